"""Seeded synthetic coupled-channel problems (inputs only).

This module draws the physics inputs of a coupled-channel scattering problem
and evaluates the user-supplied local potential at given radii.  It holds none
of the R-matrix method's arithmetic (no mesh, no kinetic matrix, no solve, no
asymptotics): both the CPU oracle and the GPU harness call it, each with radii
from its own Lagrange mesh.

The paper benchmarks "synthetic test matrices with the same block structure"
as physical problems (Sec. 5, performance results) without publishing the
generator; the recipe here follows the block structure of Eq. (block_structure)
in Sec. 2:

* channel alpha has orbital momentum l_alpha = alpha mod 4 and threshold
  E_alpha, with E_0 = 0 (entrance channel) and E_alpha ~ U(0, 5) MeV;
* the diagonal potential is a complex Woods-Saxon
  V(r) = (V0 + i W) / (1 + exp((r - R0)/ad));
* channel couplings use a derivative-Woods-Saxon form factor
  V_{alpha alpha'}(r) = s_{alpha alpha'} * 4 e^z / (1 + e^z)^2, z = (r - R0)/ad,
  with real symmetric strengths s ~ U(-5, 5) MeV drawn for alpha < alpha'.

Draw order from ``numpy.random.default_rng(seed)``: the nch-1 thresholds, then
the strict upper triangle of s in row-major order.

Charged channels (``charged_problem``) add the Coulomb interaction of a
uniformly charged sphere of radius Rc to each diagonal potential,
V_C(r) = zz_c / r for r >= Rc and zz_c (3 - r^2/Rc^2) / (2 Rc) inside, with
zz_c = Z1 Z2 e^2 (MeV fm) per channel, and leave the asymptotic region to the
Coulomb functions (Sommerfeld parameter eta_c = zz_c / (2 hm k_c)).  The
recipe follows the paper's charged-particle validation case, alpha + 208Pb
elastic scattering at E_cm = 10-50 MeV with l up to 20 (Sec. 5, physical
validation): reduced mass 4*208/212 amu, Z1 Z2 = 2*82, a generic complex
Woods-Saxon in place of the published optical potential.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HM_1AMU = 20.9  # hbar^2 / 2 mu in MeV fm^2 for a reduced mass of 1 amu
E2 = 1.44       # e^2 in MeV fm


@dataclass
class CCProblem:
    """One coupled-channel system: N = nch * nlag unknowns, nch right-hand sides."""

    nch: int
    nlag: int
    E: float                      # total energy, MeV
    l: np.ndarray                 # (nch,) int32 orbital momenta
    thresh: np.ndarray            # (nch,) float64 channel thresholds, MeV
    s: np.ndarray                 # (nch, nch) float64 coupling strengths, MeV, symmetric, zero diagonal
    a: float = 15.0               # channel radius, fm
    hm: float = HM_1AMU           # hbar^2/2mu, MeV fm^2
    V0: float = -50.0             # real WS depth, MeV
    W: float = -10.0              # imaginary WS depth, MeV (W < 0 absorbs)
    R0: float = 4.0               # WS radius, fm
    ad: float = 0.65              # WS diffuseness, fm
    bloch_B: float = 0.0          # Bloch boundary constant
    zz: np.ndarray | None = None  # (nch,) float64 Z1 Z2 e^2 per channel, MeV fm (None: neutral)
    Rc: float = 0.0               # Coulomb radius of the uniformly charged sphere, fm
    seed: int = 0
    tag: str = field(default="")

    @property
    def N(self) -> int:
        return self.nch * self.nlag


def make_problem(seed: int, nch: int, nlag: int, E: float = 10.0, *, a: float = 15.0,
                 hm: float = HM_1AMU, V0: float = -50.0, W: float = -10.0,
                 R0: float = 4.0, ad: float = 0.65, tag: str = "") -> CCProblem:
    """Draw thresholds and symmetric coupling strengths from ``seed``."""
    if nch < 1 or nlag < 1:
        raise ValueError("nch and nlag must be positive")
    rng = np.random.default_rng(seed)
    thresh = np.zeros(nch)
    if nch > 1:
        thresh[1:] = rng.uniform(0.0, 5.0, size=nch - 1)
    s = np.zeros((nch, nch))
    iu = np.triu_indices(nch, k=1)          # row-major strict upper triangle
    s[iu] = rng.uniform(-5.0, 5.0, size=iu[0].size)
    s = s + s.T
    l = (np.arange(nch) % 4).astype(np.int32)
    return CCProblem(nch=nch, nlag=nlag, E=float(E), l=l, thresh=thresh, s=s, a=a, hm=hm,
                     V0=V0, W=W, R0=R0, ad=ad, seed=seed, tag=tag)


def potential_at(p: CCProblem, r: np.ndarray) -> np.ndarray:
    """Local potential matrix at radii ``r`` (fm), in MeV.

    Returns a complex128 array of shape (nch, nch, len(r)) in C order, i.e.
    element [c2, c1, i] = V_{c1 c2}(r_i).  Its memory order is that of a
    Fortran array cpot(nr, nch, nch) (radial index fastest), the layout of the
    paper's user-supplied potential (Sec. 4, language bindings).  V is
    symmetric in (c1, c2).
    """
    r = np.asarray(r, dtype=np.float64)
    z = (r - p.R0) / p.ad
    ws = 1.0 / (1.0 + np.exp(z))
    dws = 4.0 * np.exp(z) / (1.0 + np.exp(z)) ** 2
    V = p.s[:, :, None].astype(np.complex128) * dws[None, None, :]
    diag = (p.V0 + 1j * p.W) * ws
    for c in range(p.nch):
        V[c, c, :] = diag
        if p.zz is not None and p.zz[c] != 0.0:
            V[c, c, :] += coulomb_potential(float(p.zz[c]), p.Rc, r)
    return np.ascontiguousarray(V)


def coulomb_potential(zz: float, Rc: float, r: np.ndarray) -> np.ndarray:
    """Uniformly charged sphere: zz/r outside Rc, zz (3 - r^2/Rc^2)/(2 Rc) inside (Rc=0: point)."""
    r = np.asarray(r, dtype=np.float64)
    if Rc <= 0.0:
        return zz / r
    inside = zz * (3.0 - (r / Rc) ** 2) / (2.0 * Rc)
    return np.where(r >= Rc, zz / np.maximum(r, Rc), inside)


def charged_problem(seed: int, nch: int, nlag: int, E: float = 30.0, *, a: float = 16.0,
                    Z1Z2: float = 2.0 * 82.0, mu_amu: float = 4.0 * 208.0 / 212.0,
                    V0: float = -100.0, W: float = -10.0, R0: float = 7.7, ad: float = 0.6,
                    Rc: float = 7.7, tag: str = "") -> CCProblem:
    """Charged-particle system shaped like alpha + 208Pb: thresholds and couplings
    as ``make_problem`` draws them from ``seed``, every channel charged."""
    p = make_problem(seed, nch, nlag, E, a=a, hm=HM_1AMU / mu_amu, V0=V0, W=W, R0=R0,
                     ad=ad, tag=tag)
    p.zz = np.full(nch, Z1Z2 * E2)
    p.Rc = Rc
    return p


# --- the five benchmark configurations ------------------------------------

SEEDS = {1: 11590, 2: 11591, 3: 11592, 4: 11593, 5: 11594}


def config1() -> CCProblem:
    """nch=4, nlag=50 (N=200), E=10 MeV, a=15 fm, complex WS (V0=-50, W=-10)."""
    return make_problem(SEEDS[1], 4, 50, 10.0, tag="config1")


def config2(nch: int = 256) -> CCProblem:
    """nch x nlag=100 at E=10 MeV; nch in {16, 64, 128, 256} sweeps N=1600..25600."""
    return make_problem(SEEDS[2], nch, 100, 10.0, tag=f"config2-nch{nch}")


def config3(nch: int = 256, W: float = -10.0) -> CCProblem:
    """As config 2 with its own seed; W=-1 gives the worse-conditioned case 3b."""
    return make_problem(SEEDS[3], nch, 100, 10.0, W=W, tag=f"config3-nch{nch}-W{W:g}")


def config5(E: float = 5.0) -> CCProblem:
    """nch=512, nlag=100 (N=51200); the energy sweep uses E in linspace(5, 40, 8)."""
    return make_problem(SEEDS[5], 512, 100, E, tag=f"config5-E{E:g}")


CONFIG5_ENERGIES = tuple(float(e) for e in np.linspace(5.0, 40.0, 8))


def batch_problems(n: int = 512, seed: int = SEEDS[4]) -> list[CCProblem]:
    """Config 4: n independent systems of uneven size.

    A master generator draws, per system, nch from {2,4,8,16,32,64}, nlag from
    {40,60,80,100}, E ~ U(1, 50) MeV and a per-system seed; each system's
    thresholds and couplings then come from ``make_problem`` with that seed.
    """
    master = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nch = int(master.choice([2, 4, 8, 16, 32, 64]))
        nlag = int(master.choice([40, 60, 80, 100]))
        E = float(master.uniform(1.0, 50.0))
        sub = int(master.integers(0, 2**31 - 1))
        out.append(make_problem(sub, nch, nlag, E, tag=f"batch{k}"))
    return out


# --- dense test matrices (not R-matrix systems) -----------------------------

def prescribed_kappa_hermitian(seed: int, n: int, kappa: float, nrhs: int = 1):
    """Hermitian matrix with 2-norm condition number ``kappa`` and x_exact = 1.

    Built as H D H with H = I - 2 v v^H / (v^H v) a Householder reflector and D
    a real diagonal graded geometrically from 1 to 1/kappa with alternating
    signs, the test matrices of the paper's conditioning study (Fig. illcond).
    Returns (A, B, X_exact) with B = A X_exact, all complex128 C-order.
    """
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    d = np.geomspace(1.0, 1.0 / kappa, n) * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    vv = np.vdot(v, v).real
    H = np.eye(n, dtype=np.complex128) - 2.0 * np.outer(v, v.conj()) / vv
    A = (H * d[None, :]) @ H
    X = np.ones((n, nrhs), dtype=np.complex128)
    B = A @ X
    return np.ascontiguousarray(A), np.ascontiguousarray(B), X


def random_dense(seed: int, n: int, nrhs: int = 1, dtype=np.complex128):
    """Dense complex Gaussian test matrix and right-hand sides (pivoting exercised)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    return A.astype(dtype), B.astype(dtype)
