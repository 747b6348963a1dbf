// klb_aux_f32.cu -- FP32 instantiations of the auxiliary kernels, and the
// diagnostics finalisation (precision independent).
#include "klb_aux.cuh"

namespace fdlb {

KLB_AUX_INST(float)

// One block folds all partial records, in record order per thread and a fixed
// tree across threads.
__device__ __forceinline__ void fold_records(const double* __restrict__ partials, int nparts,
                                             double* __restrict__ ring, int cap, long long* __restrict__ counter,
                                             int* __restrict__ err) {
    __shared__ double red[256][8];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double x = partials[8ll * i + k];
            acc[k] = (k == 4 || k == 5 || k == 7) ? fmax(acc[k], x) : acc[k] + x;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const double x = red[threadIdx.x + w][k];
                red[threadIdx.x][k] =
                    (k == 4 || k == 5 || k == 7) ? fmax(red[threadIdx.x][k], x) : red[threadIdx.x][k] + x;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long n = *counter;
        const long long slot = 7 * (n % cap);
        for (int k = 0; k < 7; ++k) {
            KLB_GUARD(slot + k, 7ll * cap) ring[slot + k] = red[0][k];
        }
        *counter = n + 1;
        if (red[0][7] != 0.0) atomicOr(err, ERR_NONFINITE);
    }
}

__global__ void __launch_bounds__(256) diag_finalize_kernel(const double* __restrict__ partials, int nparts,
                                                            double* __restrict__ ring, int cap,
                                                            long long* __restrict__ counter, int* __restrict__ err) {
    fold_records(partials, nparts, ring, cap, counter, err);
}

// the folds of the due members of a batch, one block each
__global__ void __launch_bounds__(256) diag_finalize_batch_kernel(const DiagJob* __restrict__ jobs, const DueMask due) {
    const int j = blockIdx.x;
    if (!KLB_DUE_BIT(due, j)) return;  // uniform across the block
    const DiagJob& J = jobs[j];
    fold_records(J.partials, J.grid, J.ring, J.cap, J.counter, J.err);
}

cudaError_t launch_diag_finalize_batch(const DiagJob* jobs, int njobs, DueMask due, cudaStream_t s) {
    if (njobs < 1) return cudaSuccess;
    diag_finalize_batch_kernel<<<njobs, 256, 0, s>>>(jobs, due);
    return cudaGetLastError();
}

KLB_BOUNDS_QUERY(bounds_flag_aux_f32)

#ifdef KLB_CHECK_BOUNDS
// self-test of the bounds-checked build: a store one element past the end of
// a buffer of n elements, which the guard skips and flags
__global__ void bounds_probe_kernel(float* p, long long n) {
    KLB_GUARD(n, n) p[n] = 0.f;
}
#endif

cudaError_t launch_bounds_probe(float* p, long long n, cudaStream_t s) {
#ifdef KLB_CHECK_BOUNDS
    bounds_probe_kernel<<<1, 1, 0, s>>>(p, n);
    return cudaGetLastError();
#else
    (void)p;
    (void)n;
    (void)s;
    return cudaErrorNotSupported;  // ordinary builds have no guard: never launched
#endif
}

cudaError_t launch_diag_finalize(const double* partials, int nparts, double* ring, int cap, long long* counter,
                                 int* err, cudaStream_t s) {
    diag_finalize_kernel<<<1, 256, 0, s>>>(partials, nparts, ring, cap, counter, err);
    return cudaGetLastError();
}

}  // namespace fdlb
