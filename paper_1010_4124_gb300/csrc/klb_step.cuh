// klb_step.cuh -- the fused FDLB time step in FP64, the parity path
// (instantiated by klb_step_f64.cu; the FP32 production step is
// klb_step_f32.cuh).
//
// One launch = one forward-Euler step (Eq. 47 of arXiv:1010.4124) over the
// whole grid.  Each CTA owns a TX x TY tile of interior nodes:
//   1. one thread issues a single 3-D TMA box load of all 19 planes of the
//      tile plus a 3-node halo (4 on the x sides so that the box starts on a
//      16-byte boundary) into shared memory, completing on an mbarrier that
//      every thread waits on with a bounded spin;
//   2. each thread takes the 19 values of its node, forms rho, u, T
//      (Eq. 10), F_k(T) (Eqs. 44-46) and the equilibrium factors (Eq. 28);
//   3. for every velocity q (unrolled; upwind side fixed at compile time),
//      each thread computes the face flux (WENO5, or the scheme chosen) of its left x-face and bottom
//      y-face from shared memory, two warps compute the tile's right and top
//      edge faces, the faces go through shared memory, and each thread forms
//      the flux divergence, the BGK term and the new value, storing it
//      (coalesced) into the other ping-pong buffer;
//   4. nodes next to a periodic or outflow side also write their ghost images
//      in the output buffer, so the next launch finds its ghosts filled;
//   5. optionally, the CTA reduces the diagnostics of its input nodes in FP64
//      to one partial record (finished by klb_diag_finalize).
#pragma once
#include "klb_device.cuh"
#include "klb_launch.h"

namespace fdlb {

template <typename T>
struct StepTile;
template <>
struct StepTile<double> {
    static constexpr int TX = 32, TY = 8;
};

template <typename T, int TX, int TY>
struct SmemLayout {
    static constexpr int SX = TX + 8;  // box width: 4 halo columns each side
    static constexpr int SY = TY + 6;  // box height: 3 halo rows each side
    static constexpr int PLANE = SX * SY;
    static constexpr size_t TILE_BYTES = sizeof(T) * NQ * PLANE;
    static constexpr int HX = TY * (TX + 1);  // x faces of the tile
    static constexpr int HY = (TY + 1) * TX;  // y faces
    static constexpr size_t BYTES = TILE_BYTES + sizeof(T) * (HX + HY);
};

// The face flux of the scheme c.scheme from the five upwind-ordered stencil
// values of F = v f (Eqs. 48-55 for WENO5; the lower-order schemes of Fig. 2:
// first-order upwind c, second-order upwind c + (c - b)/2, TVD
// c + minmod(c - b, d - c)/2), each operation as the oracle writes it.
template <typename T>
__device__ __forceinline__ T face_flux(int scheme, T a, T b, T c, T d, T e, T eps) {
    switch (scheme) {
    case 1: return c;
    case 2: return c + T(0.5) * (c - b);
    case 3: return c + T(0.5) * minmod(c - b, d - c);
    default: return Arith<T>::weno(a, b, c, d, e, eps);
    }
}
// x-face between smem columns sx-1 and sx of row sy, plane P, for the
// velocity component v of sign SGN: the flux of F = v f exactly as Eq. (48)
// states it.
template <typename T, int SX, int SGN>
__device__ __forceinline__ T face_x(const T* P, int sy, int sx, T v, T eps, int scheme) {
    const T* r = P + sy * SX;
    if (SGN > 0)
        return face_flux(scheme, v * r[sx - 3], v * r[sx - 2], v * r[sx - 1], v * r[sx], v * r[sx + 1], eps);
    return face_flux(scheme, v * r[sx + 2], v * r[sx + 1], v * r[sx], v * r[sx - 1], v * r[sx - 2], eps);
}
// y-face between smem rows sy-1 and sy of column sx, plane P.
template <typename T, int SX, int SGN>
__device__ __forceinline__ T face_y(const T* P, int sy, int sx, T v, T eps, int scheme) {
    const T* c = P + sx;
    if (SGN > 0)
        return face_flux(scheme, v * c[(sy - 3) * SX], v * c[(sy - 2) * SX], v * c[(sy - 1) * SX], v * c[sy * SX],
                         v * c[(sy + 1) * SX], eps);
    return face_flux(scheme, v * c[(sy + 2) * SX], v * c[(sy + 1) * SX], v * c[sy * SX], v * c[(sy - 1) * SX],
                     v * c[(sy - 2) * SX], eps);
}

// The shared-memory face buffers carry values between threads across
// __syncthreads(), so they must not be declared __restrict__: that would let
// the compiler reuse a neighbour's face loaded for the previous velocity.
template <typename T, int TX, int TY, int Q>
__device__ __forceinline__ void velocity_update(const StepConst<T>& c, const Geom& g, const T* tile,
                                                T* hx, T* hy, const NodeEq<T>& s,
                                                T fq, int tx, int ty, int ix, int iy, bool active,
                                                T* __restrict__ out) {
    using L = SmemLayout<T, TX, TY>;
    constexpr int SX = L::SX;
    constexpr int SGX = sgn_x(Q), SGY = sgn_y(Q);
    static_assert(std::is_same<T, double>::value, "the FP32 step is klb_step_f32.cuh");
    const T* P = tile + Q * L::PLANE;
    const int sx = tx + 4, sy = ty + 3;
    const int tid = threadIdx.x;
    const T epsx = c.eps, epsy = c.eps;
    T hl = 0, hb = 0;
    if (SGX != 0) {
        hl = face_x<T, SX, SGX>(P, sy, sx, c.vx[Q], epsx, c.scheme);
        hx[ty * (TX + 1) + tx] = hl;
    }
    if (SGY != 0) {
        hb = face_y<T, SX, SGY>(P, sy, sx, c.vy[Q], epsy, c.scheme);
        hy[ty * TX + tx] = hb;
    }
    // tile edge faces: warp 0 the top row of y faces, warp 1 the right column of x faces
    if (SGY != 0 && tid < TX) hy[TY * TX + tid] = face_y<T, SX, SGY>(P, TY + 3, tid + 4, c.vy[Q], epsy, c.scheme);
    if (SGX != 0 && tid >= 32 && tid < 32 + TY) {
        int r = tid - 32;
        hx[r * (TX + 1) + TX] = face_x<T, SX, SGX>(P, r + 3, TX + 4, c.vx[Q], epsx, c.scheme);
    }
    __syncthreads();
    // Eq. (47) as written: f - dt (dh_x/dx + dh_y/dy) - (dt/tau)(f - f^(0))
    const T dhx = SGX != 0 ? hx[ty * (TX + 1) + tx + 1] - hl : T(0);
    const T dhy = SGY != 0 ? hy[(ty + 1) * TX + tx] - hb : T(0);
    const T fn = fq - c.dt * (dhx / c.dx + dhy / c.dy) - c.relax * (fq - Arith<T>::feq(c, s, Q));
    if (active) store_with_images(out, g, Q, ix, iy, fn);
    __syncthreads();
}

template <typename T, int TX, int TY, int Q>
struct VelLoop {
    __device__ __forceinline__ static void run(const StepConst<T>& c, const Geom& g, const T* tile, T* hx, T* hy,
                                               const NodeEq<T>& s, const T* f, int tx, int ty, int ix, int iy,
                                               bool active, T* out) {
        velocity_update<T, TX, TY, Q>(c, g, tile, hx, hy, s, f[Q], tx, ty, ix, iy, active, out);
        VelLoop<T, TX, TY, Q + 1>::run(c, g, tile, hx, hy, s, f, tx, ty, ix, iy, active, out);
    }
};
template <typename T, int TX, int TY>
struct VelLoop<T, TX, TY, NQ> {
    __device__ __forceinline__ static void run(const StepConst<T>&, const Geom&, const T*, T*, T*,
                                               const NodeEq<T>&, const T*, int, int, int, int, bool, T*) {}
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) step_kernel(const __grid_constant__ CUtensorMap in_map,
                                                      const __grid_constant__ StepConst<T> c, const Geom g,
                                                      T* __restrict__ out, double* __restrict__ diag_partials,
                                                      int* __restrict__ err, long long spin_limit, int inject) {
    using L = SmemLayout<T, TX, TY>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 128 spare bytes are reserved so that the TMA destination starts on a
    // 128-byte boundary of the shared window
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    T* tile = reinterpret_cast<T*>(base);
    T* hx = reinterpret_cast<T*>(base + L::TILE_BYTES);
    T* hy = hx + L::HX;
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t never;  // fault injection: a barrier nothing arrives on

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_init(smem_u32(&never), 1);
        fence_barrier_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(b, (uint32_t)L::TILE_BYTES);
        // box origin: interior (x0 - 4, y0 - 3) = array (x0, y0); all planes
        tma_load_3d(smem_u32(tile), &in_map, x0, y0, 0, b);
    }
    __syncthreads();
    // the verdict of the bounded wait is made uniform across the CTA
    bool late = !mbar_wait_bounded(b, 0, spin_limit);
    if (inject) late = late || !mbar_wait_bounded(smem_u32(&never), 0, spin_limit);
    if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
        // let the copy in flight land before the CTA releases its shared memory
        mbar_wait_bounded(b, 0, kDrainPolls);
        return;
    }

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int ix = x0 + tx, iy = y0 + ty;
    const bool active = ix < g.nx && iy < g.ny;
    const int sx = tx + 4, sy = ty + 3;

    T f[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) f[q] = tile[q * L::PLANE + sy * L::SX + sx];
    NodeEq<T> s = Arith<T>::node_state(c, f);

    if (diag_partials != nullptr) {
        double v[8];
        node_diag(s, active, v);
        diag_block_reduce<TX * TY>(v, diag_partials + 8ll * (blockIdx.y * gridDim.x + blockIdx.x));
    }

    VelLoop<T, TX, TY, 0>::run(c, g, tile, hx, hy, s, f, tx, ty, ix, iy, active, out);
}

template <typename T>
cudaError_t launch_step_impl(const CUtensorMap& in_map, const StepConst<T>& c, const Geom& g, T* out,
                             double* diag_partials, int* err, long long spin_limit, int inject,
                             cudaStream_t stream) {
    using TT = StepTile<T>;
    constexpr int TX = TT::TX, TY = TT::TY;
    const size_t smem = SmemLayout<T, TX, TY>::BYTES + 128;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    step_kernel<T, TX, TY><<<grid, TX * TY, smem, stream>>>(in_map, c, g, out, diag_partials, err, spin_limit,
                                                            inject);
    return cudaGetLastError();
}

}  // namespace fdlb
