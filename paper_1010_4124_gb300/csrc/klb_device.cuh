// klb_device.cuh -- device-side building blocks of the FDLB step for sm_103a:
// the velocity set, the two arithmetic paths (FP32 production, FP64 parity),
// ghost images, diagnostics partials, and the TMA / mbarrier primitives.
//
// Method: Gan, Xu, Zhang & Li, arXiv:1010.4124, Secs. II-III.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
// converted to the arithmetic type T.  Both arithmetic paths read from it.
template <typename T>
struct StepConst {
    T vx[NQ], vy[NQ];  // velocity components (Eq. 5)
    T v2[NQ];          // |v_q|^2
    // FP32 path
    T cx[NQ], cy[NQ];  // dt * v_qx / dx, dt * v_qy / dy
    T ex[NQ], ey[NQ];  // WENO epsilon of the unscaled plane: eps / v_qx^2, eps / v_qy^2
    T fk[3][3];        // F_k(T) = T (fk[k][0] + T (fk[k][1] + T fk[k][2])), k = 1..3
    T ginv[4][4];      // inverse Gram matrix of the collision invariants (1, v_x, v_y, |v|^2)
    // FP64 path (the paper's formulas term by term)
    T a4[3], pk[3], den[3];  // 4 (a_{k+1} + a_{k+2}), a_{k+1} a_{k+2}, 3 a_k (a_k - a_{k+1})(a_k - a_{k+2})
    T dt, dx, dy, eps;
    T relax;  // dt / tau
};

struct Geom {
    int nx, ny;          // interior size
    int px;              // row pitch (elements)
    long long plane;     // plane stride (elements)
    int bcx_lo, bcx_hi, bcy_lo, bcy_hi;  // 0 periodic, 1 outflow, 2 fixed
};

// Macroscopic state of one node and the equilibrium factors derived from it.
template <typename T>
struct NodeEq {
    T rho, ux, uy, Tm;
    T A;      // 1 - u^2 / (2T)
    T a, b;   // u_x / T, u_y / T (FP32 path)
    T rF[4];  // rho F_k
};

// ===========================================================================
// FP32 production arithmetic.
// ===========================================================================
struct ArithF32 {
    using T = float;

    // Eqs. (44)-(46): F_k = T (p_k - 4 s_k T + 24 T^2) / den_k by Horner,
    // F_0 = 1 - 6 (F_1 + F_2 + F_3).
    __device__ __forceinline__ static void global_coeffs(const StepConst<T>& c, T Tm, T F[4]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) F[k + 1] = Tm * (c.fk[k][0] + Tm * (c.fk[k][1] + Tm * c.fk[k][2]));
        F[0] = 1.f - 6.f * (F[1] + F[2] + F[3]);
    }
    // Eq. (10) with E = sum f |v|^2 / 2 and T = E / rho - |u|^2 / 2.
    __device__ __forceinline__ static NodeEq<T> node_state(const StepConst<T>& c, const T f[NQ]) {
        T r = 0, jx = 0, jy = 0, e = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            r += f[q];
            jx += f[q] * c.vx[q];
            jy += f[q] * c.vy[q];
            e += f[q] * c.v2[q];
        }
        const T ir = 1.f / r;
        const T ux = jx * ir, uy = jy * ir;
        return from_moments(c, r, ux, uy, 0.5f * e * ir - 0.5f * (ux * ux + uy * uy));
    }
    __device__ __forceinline__ static NodeEq<T> from_moments(const StepConst<T>& c, T r, T ux, T uy, T Tm) {
        NodeEq<T> s;
        s.rho = r;
        s.ux = ux;
        s.uy = uy;
        s.Tm = Tm;
        const T u2 = ux * ux + uy * uy;
        const T iT = 1.f / Tm;
        s.A = 1.f - 0.5f * u2 * iT;
        s.a = ux * iT;
        s.b = uy * iT;
        T F[4];
        global_coeffs(c, Tm, F);
#pragma unroll
        for (int k = 0; k < 4; ++k) s.rF[k] = r * F[k];
        return s;
    }
    // Eq. (28): f^(0) = rho F_k [A + A w + w^2/2 + w^3/6], w = v.u/T.
    __device__ __forceinline__ static T feq(const StepConst<T>& c, const NodeEq<T>& s, int q) {
        const T w = c.vx[q] * s.a + c.vy[q] * s.b;
        const T br = s.A + s.A * w + w * w * (0.5f + w * (1.f / 6.f));
        return s.rF[ring_of(q)] * br;
    }
    // WENO5 flux on the unscaled plane (eps already divided by v^2), over a
    // common denominator: h = c + sum delta_q g_q P_q / sum delta_q P_q with
    // g_q = h_q - c (Eqs. 49-51) and P_q the product of the other two
    // (eps + sigma)^2 (Eqs. 52-55); one division instead of four.  Since
    // every term scales with v except the absolute epsilon,
    // h(v f; eps) = v h(f; eps / v^2): the factor v sits in the update.
    __device__ __forceinline__ static T weno(T a, T b, T c, T d, T e, T eps) {
        const T k13 = 13.f / 12.f;
        const T t1 = a - 2.f * b + c, r1 = a - 4.f * b + 3.f * c;
        const T t2 = b - 2.f * c + d, r2 = b - d;
        const T t3 = c - 2.f * d + e, r3 = 3.f * c - 4.f * d + e;
        const T s1 = eps + k13 * t1 * t1 + 0.25f * r1 * r1;
        const T s2 = eps + k13 * t2 * t2 + 0.25f * r2 * r2;
        const T s3 = eps + k13 * t3 * t3 + 0.25f * r3 * r3;
        const T p1 = s1 * s1, p2 = s2 * s2, p3 = s3 * s3;
        const T p23 = p2 * p3, p13 = p1 * p3, p12 = p1 * p2;
        const T g1 = (2.f * a - 7.f * b + 5.f * c) * (1.f / 6.f);
        const T g2 = (2.f * d - b - c) * (1.f / 6.f);
        const T g3 = (5.f * d - 4.f * c - e) * (1.f / 6.f);
        const T num = 0.1f * g1 * p23 + 0.6f * g2 * p13 + 0.3f * g3 * p12;
        const T den = 0.1f * p23 + 0.6f * p13 + 0.3f * p12;
        return c + __fdividef(num, den);
    }
    // BGK relaxation of all 19 planes in place: f_q <- f_q - (dt/tau) d_q with
    // d = f - f^(0).  In exact arithmetic d carries no mass, momentum or
    // energy (Eqs. 10-12); in FP32 the rounding of f^(0) leaves a small,
    // state-dependent residual that would accumulate step after step, so the
    // residual is projected out: d' = d - B^T (B B^T)^{-1} B d with
    // B = (1, v_x, v_y, |v|^2).  The projection changes nothing in exact
    // arithmetic and keeps the collision conservative to the rounding of d.
    __device__ __forceinline__ static void collide(const StepConst<T>& c, const NodeEq<T>& s, T f[NQ]) {
        T d[NQ];
        T m0 = 0, mx = 0, my = 0, me = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            d[q] = f[q] - feq(c, s, q);
            m0 += d[q];
            mx += d[q] * c.vx[q];
            my += d[q] * c.vy[q];
            me += d[q] * c.v2[q];
        }
        T lam[4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
            lam[a] = c.ginv[a][0] * m0 + c.ginv[a][1] * mx + c.ginv[a][2] * my + c.ginv[a][3] * me;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const T dq = d[q] - (lam[0] + lam[1] * c.vx[q] + lam[2] * c.vy[q] + lam[3] * c.v2[q]);
            f[q] = f[q] - c.relax * dq;
        }
    }
};

// ===========================================================================
// FP64 parity arithmetic: the paper's formulas evaluated term by term in the
// order in which they are written (moments Eq. 10 with T from the centred
// second moment, F_k Eqs. 44-46, f^(0) Eq. 28, the WENO5 flux of F = v f with
// four divisions Eqs. 48-55, the update Eq. 47).  The translation units that
// instantiate it are compiled with -fmad=false, so every operation is one
// IEEE-rounded step; a plain CPU evaluation of the same formulas in the same
// order therefore agrees to the last bit or close to it.
// ===========================================================================
struct ArithF64 {
    using T = double;

    __device__ __forceinline__ static void global_coeffs(const StepConst<T>& c, T Tm, T F[4]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T num = 24.0 * Tm * Tm * Tm - c.a4[k] * Tm * Tm + c.pk[k] * Tm;
            F[k + 1] = num / c.den[k];
        }
        F[0] = 1.0 - 6.0 * (F[1] + F[2] + F[3]);
    }
    __device__ __forceinline__ static NodeEq<T> node_state(const StepConst<T>& c, const T f[NQ]) {
        T r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            r += f[q];
            jx += f[q] * c.vx[q];
            jy += f[q] * c.vy[q];
        }
        const T u = jx / r, w = jy / r;
        T e = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const T cx = c.vx[q] - u, cy = c.vy[q] - w;
            e += f[q] * (cx * cx + cy * cy) / 2.0;
        }
        return from_moments(c, r, u, w, e / r);
    }
    __device__ __forceinline__ static NodeEq<T> from_moments(const StepConst<T>& c, T r, T ux, T uy, T Tm) {
        NodeEq<T> s;
        s.rho = r;
        s.ux = ux;
        s.uy = uy;
        s.Tm = Tm;
        const T u2 = ux * ux + uy * uy;
        s.A = 1.0 - u2 / (2.0 * Tm);
        s.a = 0.0;
        s.b = 0.0;
        T F[4];
        global_coeffs(c, Tm, F);
#pragma unroll
        for (int k = 0; k < 4; ++k) s.rF[k] = r * F[k];
        return s;
    }
    __device__ __forceinline__ static T feq(const StepConst<T>& c, const NodeEq<T>& s, int q) {
        const T Tm = s.Tm, A = s.A;
        const T vu = c.vx[q] * s.ux + c.vy[q] * s.uy;
        const T bracket = A + (vu / Tm) * A + (vu * vu) / (2.0 * Tm * Tm) + (vu * vu * vu) / (6.0 * Tm * Tm * Tm);
        return s.rF[ring_of(q)] * bracket;
    }
    // WENO5 flux of the already scaled stencil F = v f (Eqs. 48-55).
    __device__ __forceinline__ static T weno(T a, T b, T c, T d, T e, T eps) {
        const T h1 = (1.0 / 3.0) * a - (7.0 / 6.0) * b + (11.0 / 6.0) * c;
        const T h2 = -(1.0 / 6.0) * b + (5.0 / 6.0) * c + (1.0 / 3.0) * d;
        const T h3 = (1.0 / 3.0) * c + (5.0 / 6.0) * d - (1.0 / 6.0) * e;
        const T t1 = a - 2.0 * b + c, r1 = a - 4.0 * b + 3.0 * c;
        const T t2 = b - 2.0 * c + d, r2 = b - d;
        const T t3 = c - 2.0 * d + e, r3 = 3.0 * c - 4.0 * d + e;
        const T s1 = (13.0 / 12.0) * t1 * t1 + 0.25 * r1 * r1;
        const T s2 = (13.0 / 12.0) * t2 * t2 + 0.25 * r2 * r2;
        const T s3 = (13.0 / 12.0) * t3 * t3 + 0.25 * r3 * r3;
        const T w1 = 0.1 / ((eps + s1) * (eps + s1));
        const T w2 = 0.6 / ((eps + s2) * (eps + s2));
        const T w3 = 0.3 / ((eps + s3) * (eps + s3));
        const T ws = w1 + w2 + w3;
        return (w1 / ws) * h1 + (w2 / ws) * h2 + (w3 / ws) * h3;
    }
};

template <typename T>
using Arith = typename std::conditional<std::is_same<T, float>::value, ArithF32, ArithF64>::type;

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
