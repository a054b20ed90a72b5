// Jacobi-scaled circulant ("spectral") preconditioner for closed curves (not from the paper).
#include <cuda_runtime.h>

#include "tpe_internal.cuh"

namespace tpe {

cudaError_t spectral_setup(Ctx &c, cudaStream_t s)
{
    (void)c;
    (void)s;
    return cudaErrorNotSupported;
}

cudaError_t spectral_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip)
{
    (void)c;
    (void)r;
    (void)z;
    (void)s;
    (void)skip;
    return cudaErrorNotSupported;
}

}  // namespace tpe

extern "C" TPE_API tp_status tp_spectral_symbol(tp_ctx *ctx, int n, double *lam, tp_stream stream)
{
    (void)n;
    (void)lam;
    (void)stream;
    if (!ctx) return TP_ERR_INVALID_ARG;
    ctx->c.err = "spectral preconditioner not built";
    return TP_ERR_UNSUPPORTED;
}
