// tp_energy_static: the discrete energy of one curve network without any allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a region where allocation is not
// allowed (a host callback or a framework that forbids device allocation after start-up, an
// allocator that is being debugged, a process that has handed all free device memory to its own
// pool).  For them this entry point keeps its scratch memory (edge records, work items, partial
// sums) in fixed-size file-scope __device__ arrays that live as long as the library is loaded on a
// device.  It evaluates the same energy as tp_energy in mixed precision, for one problem (every
// ordered pair of disjoint edges of the whole graph).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "tpe_internal.cuh"

namespace tpe {
// defined in pairs.cu
cudaError_t static_energy_launch(const double *gamma, const int *edges, int nV, int nE, double alpha, double beta,
                                 double near_cutoff, RecF *recF, RecLo *recLo, double *ell, double *T, double *x,
                                 WorkItem *items, int *eslots, double *part, double *rows, int *counter, int *err,
                                 double *scal, int *off, int max_items, int max_slots, double *E, cudaStream_t s,
                                 int *status);
}  // namespace tpe

namespace {

// Scratch of the no-allocation energy, shared by every call on a device.
constexpr int kStaticMaxEdges = 65536;  // largest graph tp_energy_static accepts
constexpr int kStaticMaxItems = 8192;
constexpr int kStaticSlots = 16;

__device__ __align__(256) tpe::RecF g_recF[kStaticMaxEdges];
__device__ __align__(256) tpe::RecLo g_recLo[kStaticMaxEdges];
__device__ __align__(256) double g_ell[kStaticMaxEdges];
__device__ __align__(256) double g_T[3 * kStaticMaxEdges];
__device__ __align__(256) double g_x[3 * kStaticMaxEdges];
__device__ __align__(256) tpe::WorkItem g_items[kStaticMaxItems];
__device__ __align__(256) int g_eslots[kStaticMaxEdges];
__device__ __align__(256) double g_part[kStaticSlots * kStaticMaxEdges];
__device__ __align__(256) double g_rows[kStaticMaxEdges];
__device__ __align__(256) int g_counter[8];
__device__ __align__(256) int g_err[4];
__device__ __align__(256) double g_scal[8];
__device__ __align__(256) int g_off[4];

struct StaticPtrs {
    bool ready = false;
    tpe::RecF *recF;
    tpe::RecLo *recLo;
    double *ell, *T, *x, *part, *rows, *scal;
    tpe::WorkItem *items;
    int *eslots, *counter, *err, *off;
};

constexpr int kMaxDevices = 64;
StaticPtrs g_ptrs[kMaxDevices];
std::mutex g_mu;

template <class P, class S>
cudaError_t addr(P **out, const S &sym)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, sym);
    *out = (P *)p;
    return e;
}

// Device addresses of the scratch arrays on the current device, looked up once per device.
cudaError_t setup(StaticPtrs **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    StaticPtrs &p = g_ptrs[dev];
    if (!p.ready) {
        if ((e = addr(&p.recF, g_recF)) != cudaSuccess) return e;
        if ((e = addr(&p.recLo, g_recLo)) != cudaSuccess) return e;
        if ((e = addr(&p.ell, g_ell)) != cudaSuccess) return e;
        if ((e = addr(&p.T, g_T)) != cudaSuccess) return e;
        if ((e = addr(&p.x, g_x)) != cudaSuccess) return e;
        if ((e = addr(&p.items, g_items)) != cudaSuccess) return e;
        if ((e = addr(&p.eslots, g_eslots)) != cudaSuccess) return e;
        if ((e = addr(&p.part, g_part)) != cudaSuccess) return e;
        if ((e = addr(&p.rows, g_rows)) != cudaSuccess) return e;
        if ((e = addr(&p.counter, g_counter)) != cudaSuccess) return e;
        if ((e = addr(&p.err, g_err)) != cudaSuccess) return e;
        if ((e = addr(&p.scal, g_scal)) != cudaSuccess) return e;
        if ((e = addr(&p.off, g_off)) != cudaSuccess) return e;
        p.ready = true;
    }
    *out = &p;
    return cudaSuccess;
}

}  // namespace

extern "C" TPE_API tp_status tp_energy_static(const double *gamma, const int32_t *edges, int n_vertices,
                                              int n_edges, double alpha, double beta, double *E,
                                              tp_stream stream)
{
    if (!gamma || !E || n_vertices < 1 || n_edges < 0 || (!edges && n_edges > 0)) return TP_ERR_INVALID_ARG;
    if (n_edges > kStaticMaxEdges) return TP_ERR_INVALID_ARG;  // beyond the fixed scratch
    if (!(alpha > 1.0) || !(beta >= alpha + 2.0 - 1e-12 && beta < 2.0 * alpha + 1.0)) return TP_ERR_INVALID_ARG;
    StaticPtrs *p = nullptr;
    cudaError_t e = setup(&p);
    if (e != cudaSuccess) return TP_ERR_CUDA;
    int status = 0;
    e = tpe::static_energy_launch(gamma, edges, n_vertices, n_edges, alpha, beta, 4.0, p->recF, p->recLo, p->ell, p->T,
                                  p->x, p->items, p->eslots, p->part, p->rows, p->counter, p->err, p->scal, p->off,
                                  kStaticMaxItems, kStaticSlots, E, (cudaStream_t)stream, &status);
    if (e != cudaSuccess) return TP_ERR_CUDA;
    if (status) return (tp_status)status;  // TP_ERR_DEGENERATE_EDGE or TP_ERR_NONFINITE
    return TP_OK;
}
