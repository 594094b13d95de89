// G4 (tensor path): trailing update C22 -= L21 U12 on tcgen05 tensor cores.
// Placeholder until the tcgen05 kernel lands: the tensor precision reports an
// error instead of silently running another kernel.
#include "rmat_internal.h"

int launch_trailing_tc(rmat_ctx, float2*, int, int, int, int) { return RMAT_ESTATE; }
int tc_prepare(rmat_ctx, int, int) { return RMAT_OK; }
