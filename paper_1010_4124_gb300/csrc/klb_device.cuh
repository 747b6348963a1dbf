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

// Bounds-checked builds (-DKLB_CHECK_BOUNDS, the debug library
// libklb_checked.so): every global index a kernel forms into a state buffer,
// a dense field array or a diagnostics ring is compared with the extent of
// that buffer before the access.  An index out of range raises this
// translation unit's flag and the access is skipped (a load then reads
// zero); nothing traps, so the context stays usable and klb_sync reports
// KLB_E_BOUNDS.  Without the macro the guards expand to nothing and the
// accesses are exactly the unguarded ones.
#ifdef KLB_CHECK_BOUNDS
static __device__ int g_bounds_flag;
__device__ __forceinline__ bool idx_ok(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(&g_bounds_flag, 1);
    return false;
}
#define KLB_GUARD(i, n) if (::fdlb::idx_ok((long long)(i), (long long)(n)))
#define KLB_LOAD(p, i, n, zero) (::fdlb::idx_ok((long long)(i), (long long)(n)) ? (p)[(i)] : (zero))
// host query of this translation unit's flag (read and cleared)
#define KLB_BOUNDS_QUERY(name)                                              \
    int name() {                                                            \
        int v = 0, z = 0;                                                   \
        if (cudaMemcpyFromSymbol(&v, g_bounds_flag, sizeof(int)) != cudaSuccess) return -1; \
        if (v) cudaMemcpyToSymbol(g_bounds_flag, &z, sizeof(int));          \
        return v;                                                           \
    }
#else
#define KLB_GUARD(i, n)
#define KLB_LOAD(p, i, n, zero) ((p)[(i)])
#define KLB_BOUNDS_QUERY(name) \
    int name() { return 0; }
#endif

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
    T ex[NQ], ey[NQ];  // FP32 WENO: (3/4) eps / v_qx^2, (3/4) eps / v_qy^2 (unscaled plane, sigma scaled by 3/4)
    // the same as the pairs the packed WENO5 evaluations take, one 8-byte load
    // each: [q] = (ex, ey) of velocity q; [19 + m] = (ex, ex) of the x-only
    // velocities 6m + 3 and 6m + 6; [22 + k] = (ey, ey) of y slots 2k and 2k + 1
    alignas(8) T epair[28][2];
    T fk[3][3];        // F_k(T) = T (fk[k][0] + T (fk[k][1] + T fk[k][2])), k = 1..3
    T ginv[4][4];      // inverse Gram matrix of the collision invariants (1, v_x, v_y, |v|^2)
    // FP64 path (the paper's formulas term by term)
    T a4[3], pk[3], den[3];  // 4 (a_{k+1} + a_{k+2}), a_{k+1} a_{k+2}, 3 a_k (a_k - a_{k+1})(a_k - a_{k+2})
    T dt, dx, dy, eps;
    T relax;     // dt / tau
    int scheme;  // convection scheme (klb_scheme): 0 WENO5, 1 first-order upwind, 2 second-order upwind, 3 TVD
};

// minmod limiter of the second-order TVD scheme: the argument of smaller
// magnitude when both have the same sign, else zero
template <typename T>
__device__ __forceinline__ T minmod(T x, T y) {
    if (x > T(0) && y > T(0)) return x < y ? x : y;
    if (x < T(0) && y < T(0)) return x > y ? x : y;
    return T(0);
}

struct Geom {
    int nx, ny;          // interior size
    int px;              // row pitch (elements)
    long long plane;     // plane stride (elements)
    int bcx_lo, bcx_hi, bcy_lo, bcy_hi;  // 0 periodic, 1 outflow, 2 fixed, 3 halo (rows of another grid; no images)
};

// Macroscopic state of one node and the equilibrium factors derived from it.
template <typename T>
struct NodeEq {
    T rho, ux, uy, Tm;
    T A;      // 1 - u^2 / (2T)
    T a, b;   // u_x / T, u_y / T (FP32 path)
    T rF[4];  // rho F_k
};

// Hardware reciprocal approximation (one MUFU instruction, max error 1 ulp);
// the weights it feeds are ratios of smooth positive quantities.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// the constant pairs of the packed WENO5 flux: -1, 5/2, 11/4, -5/4, 5/6, 1/3,
// 1/2, 6, 3 (both lanes alike; see ArithF32::weno)
static __constant__ float2 kWenoPairs[9] = {{-1.f, -1.f}, {2.5f, 2.5f}, {2.75f, 2.75f}, {-1.25f, -1.25f},
                                            {5.f / 6.f, 5.f / 6.f}, {1.f / 3.f, 1.f / 3.f}, {0.5f, 0.5f},
                                            {6.f, 6.f}, {3.f, 3.f}};

// ===========================================================================
// FP32 production arithmetic.  Every operation is written as an explicitly
// rounded multiply, add or fused multiply-add, so that the compiler cannot
// contract differently in different kernels: every kernel that evaluates a
// node (either tile shape of the step, the diagnostics) gets the same bits.
// ===========================================================================
struct ArithF32 {
    using T = float;

    // Eqs. (44)-(46): F_k = T (p_k - 4 s_k T + 24 T^2) / den_k by Horner,
    // F_0 = 1 - 6 (F_1 + F_2 + F_3).
    __device__ __forceinline__ static void global_coeffs(const StepConst<T>& c, T Tm, T F[4]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) F[k + 1] = __fmul_rn(Tm, fmaf(Tm, fmaf(Tm, c.fk[k][2], c.fk[k][1]), c.fk[k][0]));
        F[0] = fmaf(-6.f, __fadd_rn(__fadd_rn(F[1], F[2]), F[3]), 1.f);
    }
    // The four collision invariants of g over the 19 velocities: sum g,
    // sum g v_x, sum g v_y, sum g |v|^2.  Within a ring, direction i + 3 is
    // -v of direction i (Eq. 5), so each ring contributes through its sum S
    // (|v|^2 is the ring's) and the three differences of opposite pairs D_i:
    //   sum g v = sum_{i=1..3} v_i D_i.
    __device__ __forceinline__ static void invariants(const StepConst<T>& c, const T g[NQ], T& m0, T& mx, T& my,
                                                      T& me) {
        m0 = g[0];
        mx = 0.f;
        my = 0.f;
        me = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 1 + 6 * k;
            const T D0 = __fsub_rn(g[b], g[b + 3]), D1 = __fsub_rn(g[b + 1], g[b + 4]);
            const T D2 = __fsub_rn(g[b + 2], g[b + 5]);
            const T S = __fadd_rn(__fadd_rn(__fadd_rn(g[b], g[b + 3]), __fadd_rn(g[b + 1], g[b + 4])),
                                  __fadd_rn(g[b + 2], g[b + 5]));
            m0 = __fadd_rn(m0, S);
            me = fmaf(c.v2[b], S, me);
            mx = fmaf(c.vx[b], D0, fmaf(c.vx[b + 1], D1, fmaf(c.vx[b + 2], D2, mx)));
            my = fmaf(c.vy[b], D0, fmaf(c.vy[b + 1], D1, my));  // directions 3 and 6 have v_y = 0
        }
    }
    // Eq. (10) with E = sum f |v|^2 / 2 and T = E / rho - |u|^2 / 2.
    __device__ __forceinline__ static NodeEq<T> node_state(const StepConst<T>& c, const T f[NQ]) {
        T r, jx, jy, e;
        invariants(c, f, r, jx, jy, e);
        const T ir = rcp_approx(r);
        const T ux = __fmul_rn(jx, ir), uy = __fmul_rn(jy, ir);
        const T u2 = fmaf(ux, ux, __fmul_rn(uy, uy));
        return from_moments(c, r, ux, uy, fmaf(__fmul_rn(0.5f, e), ir, __fmul_rn(-0.5f, u2)));
    }
    __device__ __forceinline__ static NodeEq<T> from_moments(const StepConst<T>& c, T r, T ux, T uy, T Tm) {
        NodeEq<T> s;
        s.rho = r;
        s.ux = ux;
        s.uy = uy;
        s.Tm = Tm;
        const T u2 = fmaf(ux, ux, __fmul_rn(uy, uy));
        const T iT = rcp_approx(Tm);
        s.A = fmaf(__fmul_rn(-0.5f, u2), iT, 1.f);
        s.a = __fmul_rn(ux, iT);
        s.b = __fmul_rn(uy, iT);
        T F[4];
        global_coeffs(c, Tm, F);
#pragma unroll
        for (int k = 0; k < 4; ++k) s.rF[k] = __fmul_rn(r, F[k]);
        return s;
    }
    // Eq. (28): f^(0) = rho F_k [A + A w + w^2/2 + w^3/6], w = v.u/T, written
    // as E + O with E = A + w^2/2 and O = w (A + w^2/6); direction i + 3 of a
    // ring has -w, hence E - O (the same operations as collide()).
    __device__ __forceinline__ static T feq(const StepConst<T>& c, const NodeEq<T>& s, int q) {
        if (q == 0) return __fmul_rn(s.rF[0], s.A);
        const int k = (q - 1) / 6, i = (q - 1) % 6, ib = i % 3, b = 1 + 6 * k;
        const T w = ib < 2 ? fmaf(c.vy[b + ib], s.b, __fmul_rn(c.vx[b + ib], s.a)) : __fmul_rn(c.vx[b + ib], s.a);
        const T w2 = __fmul_rn(w, w);
        const T E = fmaf(0.5f, w2, s.A);
        const T O = __fmul_rn(w, fmaf(w2, 1.f / 6.f, s.A));
        return __fmul_rn(s.rF[k + 1], i < 3 ? __fadd_rn(E, O) : __fsub_rn(E, O));
    }
    // WENO5 flux on the unscaled plane (eps already divided by v^2): with the
    // weights alpha_q = delta_q / (eps + sigma_q)^2 of Eq. (52) and the
    // candidates h_q of Eqs. (49)-(51), h = c + sum alpha_q (h_q - c) / sum alpha_q.
    // Since every term scales with v except the absolute epsilon,
    // h(v f; eps) = v h(f; eps / v^2): the factor v sits in the update.
    __device__ __forceinline__ static T weno(T a, T b, T c, T d, T e, T eps) {
        // With the differences of neighbouring values D1 = a - b (sign flipped),
        // D2 = c - b, D3 = d - c and e4 = d - e, the smoothness indicators of
        // Eqs. (53)-(55), scaled by 3/4, read
        //   s_1 = D1 (D1 + 11/4 D2) + 5/2 D2^2,
        //   s_2 = D2 (D2 - 5/4 D3) + D3^2,
        //   s_3 = e4 (e4 + 11/4 D3) + 5/2 D3^2,
        // and eps (the constant passed in) is scaled by 3/4 as well: the
        // common factor cancels in the weights.  The candidates relative to c
        // read h_1 - c = (5 D2 + 2 D1)/6, h_2 - c = (D2 + 2 D3)/6,
        // h_3 - c = (4 D3 + e4)/6; with the optimal weights delta_q and the
        // 1/6 folded in, and numerator and denominator both scaled by 10,
        //   h = c + (G1 w1 + G2 w2 + G3 w3) / (w1 + 6 w2 + 3 w3),
        //   G1 = 5/6 D2 + 1/3 D1, G2 = D2 + 2 D3, G3 = 2 D3 + e4 / 2,
        // with w_q = (1 / s_q)^2: the reciprocal of each indicator, squared
        // (the reciprocal starts as soon as the indicator is formed), and one
        // reciprocal of the sum.  Range: (1 / s_q)^2 stays a normal FP32 number
        // for 5.4e-20 <= s_q <= 9.2e18; s_q >= eps always, so eps (3/4 eps /
        // v^2 of the finest velocity component) must be at least that, and the
        // weights stay exact while the smallest indicator of a face is below
        // 9e18 (differences of f up to about 1e9).  (A common denominator of products of the
        // squared indicators, one reciprocal per face, spans s^4: it fails
        // below eps ~ 2e-10 and above differences ~ 3e4.)
        // Every operation is an explicitly rounded multiply, add or fused
        // multiply-add, in the same order as each lane of weno2(), so the
        // scalar and packed evaluations give the same bits.
        const T d1 = fmaf(b, -1.f, a), d2 = fmaf(b, -1.f, c), d3 = fmaf(c, -1.f, d), e4 = fmaf(e, -1.f, d);
        const T a2 = __fmul_rn(d2, d2), a3 = __fmul_rn(d3, d3);
        const T s1 = fmaf(d1, fmaf(2.75f, d2, d1), fmaf(2.5f, a2, eps));
        const T s2 = fmaf(d2, fmaf(-1.25f, d3, d2), fmaf(d3, d3, eps));
        const T s3 = fmaf(e4, fmaf(2.75f, d3, e4), fmaf(2.5f, a3, eps));
        const T r1 = rcp_approx(s1), r2 = rcp_approx(s2), r3 = rcp_approx(s3);
        const T w1 = __fmul_rn(r1, r1), w2 = __fmul_rn(r2, r2), w3 = __fmul_rn(r3, r3);
        const T G1 = fmaf(5.f / 6.f, d2, __fmul_rn(1.f / 3.f, d1));
        const T t3 = __fadd_rn(d3, d3);  // 2 D3, shared by G2 and G3
        const T G2 = __fadd_rn(d2, t3);
        const T G3 = fmaf(0.5f, e4, t3);
        const T num = fmaf(G1, w1, fmaf(G2, w2, __fmul_rn(G3, w3)));
        const T den = fmaf(6.f, w2, fmaf(3.f, w3, w1));
        return fmaf(num, rcp_approx(den), c);
    }
    // The same flux for two independent faces at once (packed f32x2
    // arithmetic: one instruction for both lanes of the pair; the reciprocals
    // are per lane).  Its constant pairs come from constant memory (kWenoPairs).
    __device__ __forceinline__ static float2 weno2(float2 a, float2 b, float2 c, float2 d, float2 e, float2 eps) {
        // lane by lane the same operations as weno()
        const float2 m1 = kWenoPairs[0];
        const float2 d1 = __ffma2_rn(b, m1, a), d2 = __ffma2_rn(b, m1, c);
        const float2 d3 = __ffma2_rn(c, m1, d), e4 = __ffma2_rn(e, m1, d);
        const float2 a2 = __fmul2_rn(d2, d2), a3 = __fmul2_rn(d3, d3);
        const float2 k25 = kWenoPairs[1], k275 = kWenoPairs[2];
        const float2 s1 = __ffma2_rn(d1, __ffma2_rn(k275, d2, d1), __ffma2_rn(k25, a2, eps));
        const float2 s2 = __ffma2_rn(d2, __ffma2_rn(kWenoPairs[3], d3, d2), __ffma2_rn(d3, d3, eps));
        const float2 s3 = __ffma2_rn(e4, __ffma2_rn(k275, d3, e4), __ffma2_rn(k25, a3, eps));
        const float2 r1 = make_float2(rcp_approx(s1.x), rcp_approx(s1.y));
        const float2 r2 = make_float2(rcp_approx(s2.x), rcp_approx(s2.y));
        const float2 r3 = make_float2(rcp_approx(s3.x), rcp_approx(s3.y));
        const float2 w1 = __fmul2_rn(r1, r1), w2 = __fmul2_rn(r2, r2), w3 = __fmul2_rn(r3, r3);
        const float2 G1 = __ffma2_rn(kWenoPairs[4], d2, __fmul2_rn(kWenoPairs[5], d1));
        const float2 t3 = __fadd2_rn(d3, d3);
        const float2 G2 = __fadd2_rn(d2, t3);
        const float2 G3 = __ffma2_rn(kWenoPairs[6], e4, t3);
        const float2 num = __ffma2_rn(G1, w1, __ffma2_rn(G2, w2, __fmul2_rn(G3, w3)));
        const float2 den = __ffma2_rn(kWenoPairs[7], w2, __ffma2_rn(kWenoPairs[8], w3, w1));
        const float2 r = make_float2(rcp_approx(den.x), rcp_approx(den.y));
        return __ffma2_rn(num, r, c);
    }
    // BGK relaxation of all 19 planes in place: f_q <- f_q - (dt/tau) d_q with
    // d = f - f^(0).  In exact arithmetic d carries no mass, momentum or
    // energy (Eqs. 10-12); in FP32 the rounding of f^(0) leaves a small,
    // state-dependent residual that would accumulate step after step, so the
    // residual is projected out: d' = d - B^T (B B^T)^{-1} B d with
    // B = (1, v_x, v_y, |v|^2).  The projection changes nothing in exact
    // arithmetic and keeps the collision conservative to the rounding of d.
    //
    // f^(0) is evaluated per opposite pair: with w = v.u/T for direction i,
    // direction i + 3 has -w, and the bracket splits into an even part
    // E = A + w^2/2 and an odd part O = w (A + w^2/6): br(+-w) = E +- O.
    __device__ __forceinline__ static void collide(const StepConst<T>& c, const NodeEq<T>& s, T f[NQ]) {
        T d[NQ];
        d[0] = fmaf(-s.rF[0], s.A, f[0]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 1 + 6 * k;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T w = i < 2 ? fmaf(c.vy[b + i], s.b, __fmul_rn(c.vx[b + i], s.a)) : __fmul_rn(c.vx[b + i], s.a);
                const T w2 = __fmul_rn(w, w);
                const T E = fmaf(0.5f, w2, s.A);
                const T O = __fmul_rn(w, fmaf(w2, 1.f / 6.f, s.A));
                d[b + i] = fmaf(-s.rF[k + 1], __fadd_rn(E, O), f[b + i]);
                d[b + i + 3] = fmaf(-s.rF[k + 1], __fsub_rn(E, O), f[b + i + 3]);
            }
        }
        T m0, mx, my, me;
        invariants(c, d, m0, mx, my, me);
        T lam[4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
            lam[a] = fmaf(c.ginv[a][3], me, fmaf(c.ginv[a][2], my, fmaf(c.ginv[a][1], mx, __fmul_rn(c.ginv[a][0], m0))));
        // the projection B^T lam of velocity q: lam_0 + lam_3 |v|^2 + lam_x v_x + lam_y v_y,
        // the last two odd under v -> -v
        f[0] = fmaf(-c.relax, __fsub_rn(d[0], lam[0]), f[0]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 1 + 6 * k;
            const T even = fmaf(lam[3], c.v2[b], lam[0]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T odd = i < 2 ? fmaf(lam[2], c.vy[b + i], __fmul_rn(lam[1], c.vx[b + i]))
                                    : __fmul_rn(lam[1], c.vx[b + i]);
                f[b + i] = fmaf(-c.relax, __fsub_rn(__fsub_rn(d[b + i], even), odd), f[b + i]);
                f[b + i + 3] = fmaf(-c.relax, __fadd_rn(__fsub_rn(d[b + i + 3], even), odd), f[b + i + 3]);
            }
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
// true when node (ix, iy) has ghost images to write
__device__ __forceinline__ bool has_images(const Geom& g, int ix, int iy) {
    const bool xe = g.bcx_lo == 0 ? (ix < 3 || ix >= g.nx - 3)
                                  : ((ix == 0 && g.bcx_lo == 1) || (ix == g.nx - 1 && g.bcx_hi == 1));
    const bool ye = g.bcy_lo == 0 ? (iy < 3 || iy >= g.ny - 3)
                                  : ((iy == 0 && g.bcy_lo == 1) || (iy == g.ny - 1 && g.bcy_hi == 1));
    return xe || ye;
}

template <typename T>
__device__ __forceinline__ void write_images(T* __restrict__ out, const Geom& g, int q, int ix, int iy, T val);

template <typename T>
__device__ __forceinline__ void store_with_images(T* __restrict__ out, const Geom& g, int q, int ix, int iy,
                                                  T val) {
    const long long at = (long long)q * g.plane + (long long)(iy + GY) * g.px + (ix + GX);
    KLB_GUARD(at, NQ * g.plane) out[at] = val;
    write_images(out, g, q, ix, iy, val);
}

template <typename T>
__device__ __forceinline__ void write_images(T* __restrict__ out, const Geom& g, int q, int ix, int iy, T val) {
    const long long base = (long long)q * g.plane;
    // the value at array cell (row, column) of plane q
    auto put = [&](int row, int col) {
        const long long at = base + (long long)row * g.px + col;
        KLB_GUARD(at, NQ * g.plane) out[at] = val;
    };
    // x ghost images (interior rows only)
    const bool xper = g.bcx_lo == 0;
    if (xper) {
        if (ix < 3 || ix >= g.nx - 3) {
#pragma unroll 1
            for (int m = -3; m <= 3; ++m) {
                if (m == 0) continue;
                int gxi = ix + m * g.nx;
                if ((gxi >= -3 && gxi < 0) || (gxi >= g.nx && gxi < g.nx + 3)) put(iy + GY, gxi + GX);
            }
        }
    } else {
        if (ix == 0 && g.bcx_lo == 1) {
            put(iy + GY, GX - 1);
            put(iy + GY, GX - 2);
            put(iy + GY, GX - 3);
        }
        if (ix == g.nx - 1 && g.bcx_hi == 1) {
            put(iy + GY, g.nx + GX);
            put(iy + GY, g.nx + GX + 1);
            put(iy + GY, g.nx + GX + 2);
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
                if ((gyi >= -3 && gyi < 0) || (gyi >= g.ny && gyi < g.ny + 3)) put(gyi + GY, ix + GX);
            }
        }
    } else {
        if (iy == 0 && g.bcy_lo == 1) {
            put(GY - 1, ix + GX);
            put(GY - 2, ix + GX);
            put(GY - 3, ix + GX);
        }
        if (iy == g.ny - 1 && g.bcy_hi == 1) {
            put(g.ny + GY, ix + GX);
            put(g.ny + GY + 1, ix + GX);
            put(g.ny + GY + 2, ix + GX);
        }
    }
}


// Per-node diagnostics (Sec. IV): rho, rho u_x, rho u_y, rho (T + |u|^2/2),
// |u_y|, rho u_y^2 / 2 (for the maximum), rho u_y^2 / 2 (for the sum), and a
// flag for a non-finite or non-positive rho or T.
template <typename T>
__device__ __forceinline__ void node_diag(const NodeEq<T>& s, bool active, double v[8]) {
    if (active) {
        // explicitly rounded operations: the same bits in every kernel that calls this
        double r = s.rho, u = s.ux, w = s.uy, Tm = s.Tm;
        v[0] = r;
        v[1] = __dmul_rn(r, u);
        v[2] = __dmul_rn(r, w);
        v[3] = __dmul_rn(r, __dadd_rn(Tm, __dmul_rn(0.5, __dadd_rn(__dmul_rn(u, u), __dmul_rn(w, w)))));
        v[4] = fabs(w);
        v[5] = __dmul_rn(__dmul_rn(__dmul_rn(0.5, r), w), w);
        v[6] = v[5];
        v[7] = (r > 0.0 && Tm > 0.0) ? 0.0 : 1.0;  // also catches NaN
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0;
    }
}

// The same diagnostics of an FP32 state, accumulated per thread without FP64
// work per node (FP64 runs at a small fraction of the FP32 rate on this GPU):
// the values of a node in FP32 (explicitly rounded, like the state they come
// from), each sum carried as an unevaluated pair hi + lo updated by Knuth's
// TwoSum (the rounding error of every addition is kept in lo, so the pair
// tracks the exact sum of the FP32 values to about n eps^2 relative after n
// additions), the maxima in FP32 and the flag as an integer.  A warp merges
// its threads' pairs the same way; its record (hi + lo in FP64, the layout of
// node_diag's) enters the FP64 combination across warps.
struct DiagAccF32 {
    float hi[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, lo[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float m4 = 0.f, m5 = 0.f;
    int bad = 0;
    // hi + lo <- hi + lo + x with the rounding error of hi + x carried in lo
    __device__ __forceinline__ void two_sum(int k, float x) {
        const float s = __fadd_rn(hi[k], x);
        const float xb = __fsub_rn(s, hi[k]);
        const float ha = __fsub_rn(s, xb);
        const float e = __fadd_rn(__fsub_rn(hi[k], ha), __fsub_rn(x, xb));
        hi[k] = s;
        lo[k] = __fadd_rn(lo[k], e);
    }
    __device__ __forceinline__ void add(const NodeEq<float>& s, bool active) {
        if (!active) return;
        const float r = s.rho, u = s.ux, w = s.uy, Tm = s.Tm;
        const float e = __fmul_rn(r, fmaf(0.5f, fmaf(u, u, __fmul_rn(w, w)), Tm));
        const float k = __fmul_rn(__fmul_rn(__fmul_rn(0.5f, r), w), w);
        two_sum(0, r);
        two_sum(1, __fmul_rn(r, u));
        two_sum(2, __fmul_rn(r, w));
        two_sum(3, e);
        two_sum(4, k);
        m4 = fmaxf(m4, fabsf(w));
        m5 = fmaxf(m5, k);
        bad |= (r > 0.f && Tm > 0.f) ? 0 : 1;  // also catches NaN
    }
    // hi + lo <- hi + lo + (h2 + l2): TwoSum of the leading parts, the
    // trailing parts and the rounding error added into lo
    __device__ __forceinline__ void merge(int k, float h2, float l2) {
        const float s = __fadd_rn(hi[k], h2);
        const float xb = __fsub_rn(s, hi[k]);
        const float ha = __fsub_rn(s, xb);
        const float e = __fadd_rn(__fsub_rn(hi[k], ha), __fsub_rn(h2, xb));
        hi[k] = s;
        lo[k] = __fadd_rn(__fadd_rn(lo[k], l2), e);
    }
    // the warp's accumulators combined into lane 0 (a fixed shuffle tree, so
    // deterministic), in FP32 pairs and FP32 maxima
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float h2 = __shfl_down_sync(0xffffffffu, hi[k], o);
                const float l2 = __shfl_down_sync(0xffffffffu, lo[k], o);
                merge(k, h2, l2);
            }
            m4 = fmaxf(m4, __shfl_down_sync(0xffffffffu, m4, o));
            m5 = fmaxf(m5, __shfl_down_sync(0xffffffffu, m5, o));
            bad |= __shfl_down_sync(0xffffffffu, bad, o);
        }
    }
    __device__ __forceinline__ void record(double v[8]) const {
        v[0] = __dadd_rn((double)hi[0], (double)lo[0]);
        v[1] = __dadd_rn((double)hi[1], (double)lo[1]);
        v[2] = __dadd_rn((double)hi[2], (double)lo[2]);
        v[3] = __dadd_rn((double)hi[3], (double)lo[3]);
        v[4] = m4;
        v[5] = m5;
        v[6] = __dadd_rn((double)hi[4], (double)lo[4]);
        v[7] = bad ? 1.0 : 0.0;
    }
};

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
// The same record from FP32 accumulators: the warp tree in FP32 pairs, the
// per-warp records across warps in FP64 in the order of node_diag's.
template <int NT>
__device__ __forceinline__ void diag_block_reduce(DiagAccF32 a, double* __restrict__ partial) {
    __shared__ double red[NT / 32][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a.warp_reduce();
    if (lane == 0) {
        double v[8];
        a.record(v);
#pragma unroll
        for (int k = 0; k < 8; ++k) red[w][k] = v[k];
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
