// klb_pair.cuh -- the FP32 node arithmetic of the step (moments, F_k,
// f^(0), the conservative BGK relaxation) for two nodes at once, in packed
// f32x2 arithmetic: lane x holds one node, lane y the other.  Every operation
// is, lane by lane, the explicitly rounded multiply, add or fused
// multiply-add that ArithF32 performs in the same order (a subtraction a - b
// as the fused b * (-1) + a, which rounds alike), and the reciprocals are the
// same hardware approximation per lane, so each node gets the bits ArithF32
// gives it.
#pragma once
#include "klb_device.cuh"

namespace fdlb {

// The FP32 step constants the node arithmetic needs, as (value, value) pairs:
// one 8-byte load feeds a packed operation.
struct PairConst {
    float2 vx[NQ], vy[NQ], v2[NQ];
    float2 cx[NQ], cy[NQ];  // dt v_qx / dx, dt v_qy / dy
    float2 ex[NQ], ey[NQ];  // WENO5 epsilon of the x and y planes of velocity q (3/4 eps / v^2)
    float2 fk[3][3];
    float2 ginv[4][4];
    float2 relax;
};

inline void make_pair_const(const StepConst<float>& c, PairConst& p) {
    auto P = [](float v) { return make_float2(v, v); };
    for (int q = 0; q < NQ; ++q) {
        p.vx[q] = P(c.vx[q]);
        p.vy[q] = P(c.vy[q]);
        p.v2[q] = P(c.v2[q]);
        p.cx[q] = P(c.cx[q]);
        p.cy[q] = P(c.cy[q]);
        p.ex[q] = P(c.ex[q]);
        p.ey[q] = P(c.ey[q]);
    }
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) p.fk[k][j] = P(c.fk[k][j]);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) p.ginv[a][b] = P(c.ginv[a][b]);
    p.relax = P(c.relax);
}

struct NodeEq2 {
    float2 rho, ux, uy, Tm;
    float2 A;      // 1 - u^2 / (2T)
    float2 a, b;   // u_x / T, u_y / T
    float2 rF[4];  // rho F_k
};

struct ArithF32x2 {
    static __device__ __forceinline__ float2 K(float v) { return make_float2(v, v); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, K(-1.f), a); }
    static __device__ __forceinline__ float2 rcp(float2 x) { return make_float2(rcp_approx(x.x), rcp_approx(x.y)); }

    // ArithF32::global_coeffs
    static __device__ __forceinline__ void global_coeffs(const PairConst& c, float2 Tm, float2 F[4]) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            F[k + 1] = __fmul2_rn(Tm, __ffma2_rn(Tm, __ffma2_rn(Tm, c.fk[k][2], c.fk[k][1]), c.fk[k][0]));
        F[0] = __ffma2_rn(K(-6.f), __fadd2_rn(__fadd2_rn(F[1], F[2]), F[3]), K(1.f));
    }
    // ArithF32::invariants
    static __device__ __forceinline__ void invariants(const PairConst& c, const float2 g[NQ], float2& m0, float2& mx,
                                                      float2& my, float2& me) {
        m0 = g[0];
        mx = K(0.f);
        my = K(0.f);
        me = K(0.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 1 + 6 * k;
            const float2 D0 = sub(g[b], g[b + 3]), D1 = sub(g[b + 1], g[b + 4]), D2 = sub(g[b + 2], g[b + 5]);
            const float2 S = __fadd2_rn(__fadd2_rn(__fadd2_rn(g[b], g[b + 3]), __fadd2_rn(g[b + 1], g[b + 4])),
                                        __fadd2_rn(g[b + 2], g[b + 5]));
            m0 = __fadd2_rn(m0, S);
            me = __ffma2_rn(c.v2[b], S, me);
            mx = __ffma2_rn(c.vx[b], D0, __ffma2_rn(c.vx[b + 1], D1, __ffma2_rn(c.vx[b + 2], D2, mx)));
            my = __ffma2_rn(c.vy[b], D0, __ffma2_rn(c.vy[b + 1], D1, my));
        }
    }
    // ArithF32::from_moments
    static __device__ __forceinline__ NodeEq2 from_moments(const PairConst& c, float2 r, float2 ux, float2 uy,
                                                           float2 Tm) {
        NodeEq2 s;
        s.rho = r;
        s.ux = ux;
        s.uy = uy;
        s.Tm = Tm;
        const float2 u2 = __ffma2_rn(ux, ux, __fmul2_rn(uy, uy));
        const float2 iT = rcp(Tm);
        s.A = __ffma2_rn(__fmul2_rn(K(-0.5f), u2), iT, K(1.f));
        s.a = __fmul2_rn(ux, iT);
        s.b = __fmul2_rn(uy, iT);
        float2 F[4];
        global_coeffs(c, Tm, F);
#pragma unroll
        for (int k = 0; k < 4; ++k) s.rF[k] = __fmul2_rn(r, F[k]);
        return s;
    }
    // ArithF32::node_state
    static __device__ __forceinline__ NodeEq2 node_state(const PairConst& c, const float2 f[NQ]) {
        float2 r, jx, jy, e;
        invariants(c, f, r, jx, jy, e);
        const float2 ir = rcp(r);
        const float2 ux = __fmul2_rn(jx, ir), uy = __fmul2_rn(jy, ir);
        const float2 u2 = __ffma2_rn(ux, ux, __fmul2_rn(uy, uy));
        return from_moments(c, r, ux, uy, __ffma2_rn(__fmul2_rn(K(0.5f), e), ir, __fmul2_rn(K(-0.5f), u2)));
    }
    // ArithF32::collide
    static __device__ __forceinline__ void collide(const PairConst& c, const NodeEq2& s, float2 f[NQ]) {
        const float2 m1 = K(-1.f);
        float2 d[NQ];
        d[0] = __ffma2_rn(__fmul2_rn(s.rF[0], m1), s.A, f[0]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 1 + 6 * k;
            const float2 nrF = __fmul2_rn(s.rF[k + 1], m1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float2 w = i < 2 ? __ffma2_rn(c.vy[b + i], s.b, __fmul2_rn(c.vx[b + i], s.a))
                                       : __fmul2_rn(c.vx[b + i], s.a);
                const float2 w2 = __fmul2_rn(w, w);
                const float2 E = __ffma2_rn(K(0.5f), w2, s.A);
                const float2 O = __fmul2_rn(w, __ffma2_rn(w2, K(1.f / 6.f), s.A));
                d[b + i] = __ffma2_rn(nrF, __fadd2_rn(E, O), f[b + i]);
                d[b + i + 3] = __ffma2_rn(nrF, sub(E, O), f[b + i + 3]);
            }
        }
        float2 m0, mx, my, me;
        invariants(c, d, m0, mx, my, me);
        float2 lam[4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
            lam[a] = __ffma2_rn(c.ginv[a][3], me,
                                __ffma2_rn(c.ginv[a][2], my, __ffma2_rn(c.ginv[a][1], mx, __fmul2_rn(c.ginv[a][0], m0))));
        const float2 nrelax = __fmul2_rn(c.relax, m1);
        f[0] = __ffma2_rn(nrelax, sub(d[0], lam[0]), f[0]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int b = 1 + 6 * k;
            const float2 even = __ffma2_rn(lam[3], c.v2[b], lam[0]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float2 odd = i < 2 ? __ffma2_rn(lam[2], c.vy[b + i], __fmul2_rn(lam[1], c.vx[b + i]))
                                         : __fmul2_rn(lam[1], c.vx[b + i]);
                f[b + i] = __ffma2_rn(nrelax, sub(sub(d[b + i], even), odd), f[b + i]);
                f[b + i + 3] = __ffma2_rn(nrelax, __fadd2_rn(sub(d[b + i + 3], even), odd), f[b + i + 3]);
            }
        }
    }
};

}  // namespace fdlb
