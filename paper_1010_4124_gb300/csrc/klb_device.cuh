// klb_device.cuh -- device-side building blocks of the FDLB step for sm_103a:
// the velocity set, moments, F_k(T), the truncated equilibrium, the WENO5 face
// flux, and the TMA / mbarrier primitives used by the fused step kernel.
//
// Method: Gan, Xu, Zhang & Li, arXiv:1010.4124, Secs. II-III.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdlb {

constexpr int NQ = 19;
constexpr int GX = 4;  // interior node (0, *) sits at column GX of a plane (3 ghosts + 1 pad)
constexpr int GY = 3;  // interior node (*, 0) sits at row GY (3 ghost rows)

// Error bits written to the handle's device error word.
constexpr int ERR_TIMEOUT = 1;
constexpr int ERR_NONFINITE = 2;

// Direction i = 1..6 of a ring sits at 60 i degrees (Eq. 5, N = 6).  The sign
// of each Cartesian component is fixed by the direction alone, so the upwind
// side of every face is known at compile time.
__host__ __device__ constexpr int ring_of(int q) { return q == 0 ? 0 : 1 + (q - 1) / 6; }
__host__ __device__ constexpr int dir_of(int q) { return q == 0 ? 0 : 1 + (q - 1) % 6; }
// sign of cos(60 i deg): i = 1..6 -> +, -, -, -, +, +
__host__ __device__ constexpr int sgn_x(int q) {
    return q == 0 ? 0 : (dir_of(q) == 1 || dir_of(q) == 5 || dir_of(q) == 6) ? 1 : -1;
}
// sign of sin(60 i deg): i = 1..6 -> +, +, 0, -, -, 0
__host__ __device__ constexpr int sgn_y(int q) {
    return q == 0 ? 0 : (dir_of(q) == 1 || dir_of(q) == 2) ? 1 : (dir_of(q) == 4 || dir_of(q) == 5) ? -1 : 0;
}

// Per-instance constants of the step, computed on the host in double and
// converted to the arithmetic type T.
template <typename T>
struct StepConst {
    T vx[NQ], vy[NQ];  // velocity components (Eq. 5)
    T v2[NQ];          // |v_q|^2
    T cx[NQ], cy[NQ];  // dt * v_qx / dx, dt * v_qy / dy
    T ex[NQ], ey[NQ];  // WENO epsilon of the unscaled plane: eps / v_qx^2, eps / v_qy^2
    T fk[3][3];        // F_k(T) = T (fk[k][0] + T (fk[k][1] + T fk[k][2])), k = 1..3
    T relax;           // dt / tau
};

struct Geom {
    int nx, ny;          // interior size
    int px;              // row pitch (elements)
    long long plane;     // plane stride (elements)
    int bcx_lo, bcx_hi, bcy_lo, bcy_hi;  // 0 periodic, 1 outflow, 2 fixed
};

// ---------------------------------------------------------------------------
// Global coefficients, Eqs. (44)-(46): F_k = T (p_k - 4 s_k T + 24 T^2) / den_k
// with the cyclic ring index; F_0 = 1 - 6 (F_1 + F_2 + F_3).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void global_coeffs(const StepConst<T>& c, T Tm, T F[4]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k + 1] = Tm * (c.fk[k][0] + Tm * (c.fk[k][1] + Tm * c.fk[k][2]));
    F[0] = T(1) - T(6) * (F[1] + F[2] + F[3]);
}

// Macroscopic state of one node and the equilibrium factors derived from it.
template <typename T>
struct NodeEq {
    T rho, ux, uy, Tm;
    T A;        // 1 - u^2 / (2T)
    T a, b;     // u_x / T, u_y / T
    T rF[4];    // rho F_k
};

// Eq. (10): rho = sum f, rho u = sum f v, rho T = sum f (v-u)^2/2, written as
// E = sum f |v|^2 / 2 and T = E / rho - |u|^2 / 2.
template <typename T>
__device__ __forceinline__ NodeEq<T> node_state(const StepConst<T>& c, const T f[NQ]) {
    T r = 0, jx = 0, jy = 0, e = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        r += f[q];
        jx += f[q] * c.vx[q];
        jy += f[q] * c.vy[q];
        e += f[q] * c.v2[q];
    }
    NodeEq<T> s;
    T ir = T(1) / r;
    s.rho = r;
    s.ux = jx * ir;
    s.uy = jy * ir;
    T u2 = s.ux * s.ux + s.uy * s.uy;
    s.Tm = T(0.5) * e * ir - T(0.5) * u2;
    T iT = T(1) / s.Tm;
    s.A = T(1) - T(0.5) * u2 * iT;
    s.a = s.ux * iT;
    s.b = s.uy * iT;
    T F[4];
    global_coeffs(c, s.Tm, F);
#pragma unroll
    for (int k = 0; k < 4; ++k) s.rF[k] = r * F[k];
    return s;
}

// Truncated equilibrium, Eq. (28):
//   f_q^(0) = rho F_k [A + A w + w^2/2 + w^3/6],  w = v_q . u / T.
template <typename T>
__device__ __forceinline__ T feq_q(const StepConst<T>& c, const NodeEq<T>& s, int q) {
    T w = c.vx[q] * s.a + c.vy[q] * s.b;
    T br = s.A + s.A * w + w * w * (T(0.5) + w * T(1.0 / 6.0));
    return s.rF[ring_of(q)] * br;
}

// ---------------------------------------------------------------------------
// Fifth-order WENO flux at I+1/2 (Eqs. 48-55) for one plane of f, with the
// five stencil values already in upwind order (a..e = f_{I-2..I+2} for a
// non-negative component, f_{I+3..I-1} for a negative one).  The paper applies
// the scheme to F = v f; since every term scales with v except the absolute
// epsilon, h(v f; eps) = v h(f; eps / v^2): the caller passes eps / v^2 and
// multiplies by v in the update coefficient.
//
// The convex combination is evaluated over a common denominator,
//   h = c + sum_q delta_q g_q P_q / sum_q delta_q P_q,
// with g_q = h_q - c and P_q the product of the other two (eps + sigma)^2
// terms; this is algebraically identical to Eq. (48) with Eq. (52) and needs
// one division instead of four.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T divide(T n, T d) { return n / d; }
template <>
__device__ __forceinline__ float divide<float>(float n, float d) { return __fdividef(n, d); }

template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e, T eps) {
    const T k13 = T(13.0 / 12.0);
    T t1 = a - T(2) * b + c, r1 = a - T(4) * b + T(3) * c;
    T t2 = b - T(2) * c + d, r2 = b - d;
    T t3 = c - T(2) * d + e, r3 = T(3) * c - T(4) * d + e;
    T s1 = eps + k13 * t1 * t1 + T(0.25) * r1 * r1;
    T s2 = eps + k13 * t2 * t2 + T(0.25) * r2 * r2;
    T s3 = eps + k13 * t3 * t3 + T(0.25) * r3 * r3;
    T p1 = s1 * s1, p2 = s2 * s2, p3 = s3 * s3;
    T p23 = p2 * p3, p13 = p1 * p3, p12 = p1 * p2;
    // g_q = h_q - c with h_q from Eqs. (49)-(51)
    T g1 = (T(2) * a - T(7) * b + T(5) * c) * T(1.0 / 6.0);
    T g2 = (T(2) * d - b - c) * T(1.0 / 6.0);
    T g3 = (T(5) * d - T(4) * c - e) * T(1.0 / 6.0);
    T num = T(0.1) * g1 * p23 + T(0.6) * g2 * p13 + T(0.3) * g3 * p12;
    T den = T(0.1) * p23 + T(0.6) * p13 + T(0.3) * p12;
    return c + divide(num, den);
}


// ---------------------------------------------------------------------------
// Ghost images.  A node next to a periodic side is also written to the ghost
// nodes it wraps to; the edge node next to an outflow side is copied to the
// three ghost nodes beyond it (zeroth-order extrapolation of f, Eqs. 63-64
// with the non-equilibrium part extrapolated the same way).  Fixed-equilibrium
// ghosts (Eq. 57) are written once at initialisation and never touched.
// Corner ghosts are never read by the dimension-by-dimension stencils.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void store_with_images(T* __restrict__ out, const Geom& g, int q, int ix, int iy,
                                                  T val) {
    const long long base = (long long)q * g.plane;
    out[base + (long long)(iy + GY) * g.px + (ix + GX)] = val;
    // x ghost images (interior rows only)
    const bool xper = g.bcx_lo == 0;
    if (xper) {
        if (ix < 3 || ix >= g.nx - 3) {
#pragma unroll 1
            for (int m = -3; m <= 3; ++m) {
                if (m == 0) continue;
                int gxi = ix + m * g.nx;
                if ((gxi >= -3 && gxi < 0) || (gxi >= g.nx && gxi < g.nx + 3))
                    out[base + (long long)(iy + GY) * g.px + (gxi + GX)] = val;
            }
        }
    } else {
        if (ix == 0 && g.bcx_lo == 1) {
            out[base + (long long)(iy + GY) * g.px + (GX - 1)] = val;
            out[base + (long long)(iy + GY) * g.px + (GX - 2)] = val;
            out[base + (long long)(iy + GY) * g.px + (GX - 3)] = val;
        }
        if (ix == g.nx - 1 && g.bcx_hi == 1) {
            out[base + (long long)(iy + GY) * g.px + (g.nx + GX)] = val;
            out[base + (long long)(iy + GY) * g.px + (g.nx + GX + 1)] = val;
            out[base + (long long)(iy + GY) * g.px + (g.nx + GX + 2)] = val;
        }
    }
    // y ghost images (interior columns only)
    const bool yper = g.bcy_lo == 0;
    if (yper) {
        if (iy < 3 || iy >= g.ny - 3) {
#pragma unroll 1
            for (int m = -3; m <= 3; ++m) {
                if (m == 0) continue;
                int gyi = iy + m * g.ny;
                if ((gyi >= -3 && gyi < 0) || (gyi >= g.ny && gyi < g.ny + 3))
                    out[base + (long long)(gyi + GY) * g.px + (ix + GX)] = val;
            }
        }
    } else {
        if (iy == 0 && g.bcy_lo == 1) {
            out[base + (long long)(GY - 1) * g.px + (ix + GX)] = val;
            out[base + (long long)(GY - 2) * g.px + (ix + GX)] = val;
            out[base + (long long)(GY - 3) * g.px + (ix + GX)] = val;
        }
        if (iy == g.ny - 1 && g.bcy_hi == 1) {
            out[base + (long long)(g.ny + GY) * g.px + (ix + GX)] = val;
            out[base + (long long)(g.ny + GY + 1) * g.px + (ix + GX)] = val;
            out[base + (long long)(g.ny + GY + 2) * g.px + (ix + GX)] = val;
        }
    }
}


// Per-node diagnostics (Sec. IV): rho, rho u_x, rho u_y, rho (T + |u|^2/2),
// |u_y|, rho u_y^2 / 2 (for the maximum), rho u_y^2 / 2 (for the sum), and a
// flag for a non-finite or non-positive rho or T.
template <typename T>
__device__ __forceinline__ void node_diag(const NodeEq<T>& s, bool active, double v[8]) {
    if (active) {
        double r = s.rho, u = s.ux, w = s.uy, Tm = s.Tm;
        v[0] = r;
        v[1] = r * u;
        v[2] = r * w;
        v[3] = r * (Tm + 0.5 * (u * u + w * w));
        v[4] = fabs(w);
        v[5] = 0.5 * r * w * w;
        v[6] = v[5];
        v[7] = (r > 0.0 && Tm > 0.0) ? 0.0 : 1.0;  // also catches NaN
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0;
    }
}

// Block reduction of the diagnostics (FP64) to one partial record: sums for
// slots 0-3 and 6, maxima for 4, 5 and the flag 7.  The shuffle tree and the
// warp order are fixed, so the result is deterministic.
template <int NT>
__device__ __forceinline__ void diag_block_reduce(double v[8], double* __restrict__ partial) {
    __shared__ double red[NT / 32][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            x = (k == 4 || k == 5 || k == 7) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        double x = red[0][k];
        for (int i = 1; i < NT / 32; ++i) x = (k == 4 || k == 5 || k == 7) ? fmax(x, red[i][k]) : x + red[i][k];
        partial[k] = x;
    }
}

// ---------------------------------------------------------------------------
// TMA and mbarrier primitives (inline PTX, sm_90+ / sm_103a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each poll may suspend the warp
// for a hardware-defined interval), so a lost transaction ends the kernel with
// an error status instead of a hang.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

}  // namespace fdlb
