// klb_aux.cuh -- small kernels around the step (templates; klb_aux_f32.cu and
// klb_aux_f64.cu instantiate them): initial equilibrium state,
// fixed-equilibrium ghosts, distribution import / export, macroscopic fields,
// and the diagnostics partials.  All are elementwise or single-pass
// reductions; none is on the per-step hot path.
#pragma once
#include "klb_launch.h"

namespace fdlb {

// f := f^(0)(rho, u, T) at every interior node (Eq. 28), with ghost images,
// written to buffer a (and to b when it is not NULL).  The fields may live in
// host memory the device can read (pinned, mapped).
template <typename T>
__global__ void init_feq_kernel(const StepConst<T> c, const Geom g, const double* __restrict__ rho,
                                const double* __restrict__ ux, const double* __restrict__ uy,
                                const double* __restrict__ Tm, T* __restrict__ a, T* __restrict__ b) {
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(k % g.nx), iy = (int)(k / g.nx);
        const NodeEq<T> s = Arith<T>::from_moments(c, T(rho[k]), T(ux[k]), T(uy[k]), T(Tm[k]));
#pragma unroll 1
        for (int q = 0; q < NQ; ++q) {
            const T v = Arith<T>::feq(c, s, q);
            store_with_images(a, g, q, ix, iy, v);
            if (b) store_with_images(b, g, q, ix, iy, v);
        }
    }
}

// Fixed-equilibrium ghosts (Eq. 57): the three ghost nodes beyond an edge node
// hold f^(0) of that node's initial state, for every side with FIXED_EQ.
template <typename T>
__global__ void fixed_ghosts_kernel(const StepConst<T> c, const Geom g, const double* __restrict__ rho,
                                    const double* __restrict__ ux, const double* __restrict__ uy,
                                    const double* __restrict__ Tm, T* __restrict__ a, T* __restrict__ b) {
    // items: [0, ny) x-lo rows, [ny, 2ny) x-hi rows, then nx columns y-lo, nx y-hi
    const int total = 2 * g.ny + 2 * g.nx;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int side, ix, iy;
        if (t < 2 * g.ny) {
            side = t < g.ny ? 0 : 1;
            iy = t % g.ny;
            ix = side == 0 ? 0 : g.nx - 1;
            if ((side == 0 ? g.bcx_lo : g.bcx_hi) != 2) continue;
        } else {
            const int u = t - 2 * g.ny;
            side = u < g.nx ? 2 : 3;
            ix = u % g.nx;
            iy = side == 2 ? 0 : g.ny - 1;
            if ((side == 2 ? g.bcy_lo : g.bcy_hi) != 2) continue;
        }
        const long long k = (long long)iy * g.nx + ix;
        const NodeEq<T> s = Arith<T>::from_moments(c, T(rho[k]), T(ux[k]), T(uy[k]), T(Tm[k]));
#pragma unroll 1
        for (int q = 0; q < NQ; ++q) {
            const T v = Arith<T>::feq(c, s, q);
            for (int d = 1; d <= 3; ++d) {
                long long off;
                if (side == 0) off = (long long)(iy + GY) * g.px + (GX - d);
                else if (side == 1) off = (long long)(iy + GY) * g.px + (g.nx - 1 + GX + d);
                else if (side == 2) off = (long long)(GY - d) * g.px + (ix + GX);
                else off = (long long)(g.ny - 1 + GY + d) * g.px + (ix + GX);
                KLB_GUARD(q * g.plane + off, NQ * g.plane) a[q * g.plane + off] = v;
                KLB_GUARD(q * g.plane + off, NQ * g.plane) b[q * g.plane + off] = v;
            }
        }
    }
}

template <typename T>
__global__ void set_f_kernel(const Geom g, const double* __restrict__ src, T* __restrict__ dst) {
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < NQ * n;
         k += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(k / n);
        const long long r = k % n;
        store_with_images(dst, g, q, (int)(r % g.nx), (int)(r / g.nx), T(KLB_LOAD(src, k, NQ * n, 0.0)));
    }
}

template <typename T>
__global__ void get_f_kernel(const Geom g, const T* __restrict__ src, double* __restrict__ dst) {
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < NQ * n;
         k += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(k / n);
        const long long r = k % n;
        const int ix = (int)(r % g.nx), iy = (int)(r / g.nx);
        const long long at = q * g.plane + (long long)(iy + GY) * g.px + (ix + GX);
        KLB_GUARD(k, NQ * n) dst[k] = double(KLB_LOAD(src, at, NQ * g.plane, T(0)));
    }
}

template <typename T>
__global__ void fields_kernel(const StepConst<T> c, const Geom g, const T* __restrict__ f,
                              double* __restrict__ rho, double* __restrict__ ux, double* __restrict__ uy,
                              double* __restrict__ Tm) {
    const long long n = (long long)g.nx * g.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(k % g.nx), iy = (int)(k / g.nx);
        T fl[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            fl[q] = KLB_LOAD(f, q * g.plane + (long long)(iy + GY) * g.px + (ix + GX), NQ * g.plane, T(0));
        const NodeEq<T> s = Arith<T>::node_state(c, fl);
        if (rho) rho[k] = s.rho;
        if (ux) ux[k] = s.ux;
        if (uy) uy[k] = s.uy;
        if (Tm) Tm[k] = s.Tm;
    }
}

// Diagnostics partials of a state over the same TX x TY tiles, in the same
// reduction order, as the fused path inside the step kernel.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) diag_partials_kernel(const StepConst<T> c, const Geom g,
                                                               const T* __restrict__ f,
                                                               double* __restrict__ partials) {
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int ix = blockIdx.x * TX + tx, iy = blockIdx.y * TY + ty;
    const bool active = ix < g.nx && iy < g.ny;
    T fl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        fl[q] = active ? KLB_LOAD(f, q * g.plane + (long long)(iy + GY) * g.px + (ix + GX), NQ * g.plane, T(1)) : T(1);
    const NodeEq<T> s = Arith<T>::node_state(c, fl);
    double v[8];
    node_diag(s, active, v);
    diag_block_reduce<TX * TY>(v, partials + 8ll * (blockIdx.y * gridDim.x + blockIdx.x));
}

// Averaged density profile (Sec. IV.A): rho_bar[j] = (1/nx) sum_i rho(i, j),
// the interface lying along x.  One CTA per row; rho = sum_q f_q and the row
// sum in FP64, reduced in a fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) mean_density_kernel(const Geom g, const T* __restrict__ f,
                                                           double* __restrict__ out) {
    __shared__ double part[8];
    const int j = blockIdx.x;
    const T* row = f + (long long)(j + GY) * g.px + GX;
    double s = 0.0;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            r += (double)KLB_LOAD(row, q * g.plane + i, NQ * g.plane - ((long long)(j + GY) * g.px + GX), T(0));
        s += r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        KLB_GUARD(j, g.ny) out[j] = t / g.nx;
    }
}

template <typename T>
cudaError_t launch_mean_density(const Geom& g, const T* f, double* out, cudaStream_t s) {
    mean_density_kernel<T><<<g.ny, 256, 0, s>>>(g, f, out);
    return cudaGetLastError();
}

static inline int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

template <typename T>
cudaError_t launch_init_feq(const StepConst<T>& c, const Geom& g, const double* rho, const double* ux,
                            const double* uy, const double* Tm, T* a, T* b, cudaStream_t s) {
    init_feq_kernel<T><<<grid_for((long long)g.nx * g.ny, 256), 256, 0, s>>>(c, g, rho, ux, uy, Tm, a, b);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fixed_ghosts(const StepConst<T>& c, const Geom& g, const double* rho, const double* ux,
                                const double* uy, const double* Tm, T* a, T* b, cudaStream_t s) {
    fixed_ghosts_kernel<T><<<grid_for(2ll * (g.nx + g.ny), 128), 128, 0, s>>>(c, g, rho, ux, uy, Tm, a, b);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_set_f(const Geom& g, const double* src, T* dst, cudaStream_t s) {
    set_f_kernel<T><<<grid_for(19ll * g.nx * g.ny, 256), 256, 0, s>>>(g, src, dst);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_get_f(const Geom& g, const T* src, double* dst, cudaStream_t s) {
    get_f_kernel<T><<<grid_for(19ll * g.nx * g.ny, 256), 256, 0, s>>>(g, src, dst);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fields(const StepConst<T>& c, const Geom& g, const T* f, double* rho, double* ux, double* uy,
                          double* Tm, cudaStream_t s) {
    fields_kernel<T><<<grid_for((long long)g.nx * g.ny, 256), 256, 0, s>>>(c, g, f, rho, ux, uy, Tm);
    return cudaGetLastError();
}
template <typename T, int TX, int TY>
cudaError_t launch_diag_partials_tiles(const StepConst<T>& c, const Geom& g, const T* f, double* partials,
                                       cudaStream_t s) {
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    diag_partials_kernel<T, TX, TY><<<grid, TX * TY, 0, s>>>(c, g, f, partials);
    return cudaGetLastError();
}

#define KLB_AUX_INST(T)                                                                                  \
    template cudaError_t launch_mean_density<T>(const Geom&, const T*, double*, cudaStream_t);                  \
    template cudaError_t launch_init_feq<T>(const StepConst<T>&, const Geom&, const double*, const double*,     \
                                            const double*, const double*, T*, T*, cudaStream_t);              \
    template cudaError_t launch_fixed_ghosts<T>(const StepConst<T>&, const Geom&, const double*, const double*, \
                                                const double*, const double*, T*, T*, cudaStream_t);          \
    template cudaError_t launch_set_f<T>(const Geom&, const double*, T*, cudaStream_t);                         \
    template cudaError_t launch_get_f<T>(const Geom&, const T*, double*, cudaStream_t);                         \
    template cudaError_t launch_fields<T>(const StepConst<T>&, const Geom&, const T*, double*, double*, double*, \
                                          double*, cudaStream_t);

}  // namespace fdlb
