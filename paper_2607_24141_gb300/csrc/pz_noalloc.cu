// pz_noalloc.cu -- a variant of the per-element abundance-gradient reduction that
// allocates no device memory.
//
// The regular path (pz_backward) sums the per-line oscillator-strength gradients of
// each element into FP64 accumulators that the context allocates.  Some callers
// cannot call cudaMalloc at the point where they need this reduction: a framework
// that owns every byte of device memory through its own pool (a stray cudaMalloc
// escapes its accounting or fails under its hard memory cap), or a tight optimiser
// loop that cannot accept cudaMalloc's implicit device synchronisation.  This entry
// point serves them: its accumulators are a fixed array in the library's own device
// image, so it never allocates.
//
// The array holds kNoAllocMaxElem doubles (32 KiB) on every GPU that loads the
// library, until the process exits.  Every call shares it: each call clears the
// entries it uses before summing, and two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on it and give wrong sums.
#include <cuda_runtime.h>

#include <mutex>

#include "pz_internal.h"

namespace pz {

constexpr int kNoAllocMaxElem = 4096;

// Scratch accumulators.  Device code may name the array directly; host code must use
// the address looked up with cudaGetSymbolAddress (the host-side name is only a
// stand-in, not a device address).
static __device__ __align__(256) double g_noalloc_elem_acc[kNoAllocMaxElem];

__global__ void k_noalloc_clear(double *acc, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) acc[k] = 0.0;
}

__global__ void k_noalloc_sum(const float *g, const int32_t *species, const int32_t *eos, int64_t n_lines,
                              int32_t n_species, int32_t n_elem, double *acc) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    const int32_t s = species[l];
    if (s < 0 || s >= n_species) return;
    const int32_t e = eos[s];
    if (e < 0 || e >= n_elem) return;
    atomicAdd(acc + e, (double)g[l]);
}

__global__ void k_noalloc_store(const double *acc, int n, float *out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = (float)acc[k];
}

// Device address of the scratch array, looked up once per device with that device
// current.
static pz_status scratch_address(double **out) {
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "pz_abundance_grad_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(PZ_EINVAL, "pz_abundance_grad_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_elem_acc);
        if (e != cudaSuccess) return cuda_check(e, "pz_abundance_grad_noalloc: cudaGetSymbolAddress");
        addr[dev] = static_cast<double *>(p);
    }
    *out = addr[dev];
    return PZ_OK;
}

}  // namespace pz

using namespace pz;

extern "C" pz_status pz_abundance_grad_noalloc(const float *g_dlog_gf, const int32_t *species,
                                               const int32_t *elem_of_species, int64_t n_lines, int32_t n_species,
                                               int32_t n_elem, float *g_dabund, void *stream) {
    if (n_elem < 1 || n_elem > kNoAllocMaxElem)
        return fail(PZ_EINVAL, "pz_abundance_grad_noalloc: n_elem must be in [1, 4096] (size of the fixed scratch)");
    if (n_lines < 0 || n_species < 1) return fail(PZ_EINVAL, "pz_abundance_grad_noalloc: bad n_lines or n_species");
    if (!g_dabund || !elem_of_species || (n_lines > 0 && (!g_dlog_gf || !species)))
        return fail(PZ_EINVAL, "pz_abundance_grad_noalloc: NULL pointer");
    double *acc = nullptr;
    pz_status st = scratch_address(&acc);
    if (st != PZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_clear<<<(n_elem + 255) / 256, 256, 0, s>>>(acc, n_elem);
    if (n_lines > 0)
        k_noalloc_sum<<<(unsigned)((n_lines + 255) / 256), 256, 0, s>>>(g_dlog_gf, species, elem_of_species, n_lines,
                                                                        n_species, n_elem, acc);
    k_noalloc_store<<<(n_elem + 255) / 256, 256, 0, s>>>(acc, n_elem, g_dabund);
    return cuda_check(cudaGetLastError(), "pz_abundance_grad_noalloc");
}
