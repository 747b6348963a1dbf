// klb_adjoint.cuh -- adjoint (vector-Jacobian product) of the FDLB step.
//
// For the step f^{n+1} = S(f^n) of Eq. (47) (arXiv:1010.4124) and a
// sensitivity lambda^{n+1} = dL/df^{n+1}, these kernels form
//   lambda^n = (dS/df^n)^T lambda^{n+1}
// on the interior nodes, with every dependence through ghost nodes folded back
// onto the interior node the ghost copies (periodic wrap, outflow copy).
// Three parts:
//   * faces: for each WENO5 face h (Eqs. 48-55 applied to F = v f), the
//     sensitivity mu = dL/dh = (dt/dx)(lambda(right node) - lambda(left node))
//     times the gradient of h with respect to its five stencil values,
//     nonlinear weights included, written to a face-gradient buffer;
//   * gather: each node collects, without atomics, the entries of the faces
//     whose stencils contain it or one of its ghost images, and adds the
//     adjoint of the BGK term: (1 - dt/tau) lambda + (dt/tau) (d f^(0)/df)^T lambda,
//     the latter through the four moments (rho, rho u, E) that f^(0) depends on;
//   * sources and the initial state: dK/df for K = sum rho u_y^2 / 2, and
//     (d f^(0) / d(rho, u_x, u_y, T))^T lambda^0 for the initial fields.
#pragma once
#include "klb_device.cuh"

namespace fdlb {

// 1/x: correctly rounded in FP64 (the accuracy reference of the adjoint), the
// hardware approximation in FP32 (the FP32 adjoint is checked against the FP64
// one to 2e-3)
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return rcp_approx(x); }

// F_k(T) and dF_k/dT for k = 0..3 (Eqs. 44-46 and their derivative)
template <typename T>
__device__ __forceinline__ void coeffs_and_slope(const StepConst<T>& c, T Tm, T F[4], T dF[4]) {
    T s = 0, ds = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T id = recip(c.den[k]);
        F[k + 1] = (T(24) * Tm * Tm * Tm - c.a4[k] * Tm * Tm + c.pk[k] * Tm) * id;
        dF[k + 1] = (T(72) * Tm * Tm - T(2) * c.a4[k] * Tm + c.pk[k]) * id;
        s += F[k + 1];
        ds += dF[k + 1];
    }
    F[0] = T(1) - T(6) * s;
    dF[0] = -T(6) * ds;
}

// Gradient of the WENO5 flux h(a, b, c, d, e) (Eqs. 48-55) with respect to its
// five inputs.  With alpha_q = delta_q / (eps + sigma_q)^2, S = sum alpha,
// omega_q = alpha_q / S:
//   dh/dx = sum_q omega_q dh_q/dx + sum_q beta_q dsigma_q/dx,
//   beta_q = -2 alpha_q (h_q - h) / ((eps + sigma_q) S).
template <typename T>
__device__ __forceinline__ T weno5_grad(T a, T b, T c, T d, T e, T eps, T g[5]) {
    const T r6 = T(1) / T(6);
    const T h1 = (T(2) * a - T(7) * b + T(11) * c) * r6;
    const T h2 = (-b + T(5) * c + T(2) * d) * r6;
    const T h3 = (T(2) * c + T(5) * d - e) * r6;
    const T t1 = a - T(2) * b + c, r1 = a - T(4) * b + T(3) * c;
    const T t2 = b - T(2) * c + d, r2 = b - d;
    const T t3 = c - T(2) * d + e, r3 = T(3) * c - T(4) * d + e;
    const T k13 = T(13) / T(12);
    const T s1 = eps + k13 * t1 * t1 + T(0.25) * r1 * r1;
    const T s2 = eps + k13 * t2 * t2 + T(0.25) * r2 * r2;
    const T s3 = eps + k13 * t3 * t3 + T(0.25) * r3 * r3;
    // one reciprocal per indicator and one for the sum of the alphas
    const T i1 = recip(s1), i2 = recip(s2), i3 = recip(s3);
    const T al1 = T(0.1) * i1 * i1, al2 = T(0.6) * i2 * i2, al3 = T(0.3) * i3 * i3;
    const T iS = recip(al1 + al2 + al3);
    const T w1 = al1 * iS, w2 = al2 * iS, w3 = al3 * iS;
    const T h = w1 * h1 + w2 * h2 + w3 * h3;
    const T b1 = -T(2) * w1 * (h1 - h) * i1;
    const T b2 = -T(2) * w2 * (h2 - h) * i2;
    const T b3 = -T(2) * w3 * (h3 - h) * i3;
    // dsigma_q/dx: d(13/12 t^2 + r^2/4) = 13/6 t dt + r/2 dr
    const T k136 = T(13) / T(6);
    const T u1 = k136 * t1, v1 = T(0.5) * r1;  // coefficients of dt1, dr1
    const T u2 = k136 * t2, v2 = T(0.5) * r2;
    const T u3 = k136 * t3, v3 = T(0.5) * r3;
    // t1 = a - 2b + c, r1 = a - 4b + 3c ; t2 = b - 2c + d, r2 = b - d ; t3 = c - 2d + e, r3 = 3c - 4d + e
    g[0] = w1 * (T(2) / T(6)) + b1 * (u1 + v1);
    g[1] = w1 * (-T(7) / T(6)) + w2 * (-T(1) / T(6)) + b1 * (-T(2) * u1 - T(4) * v1) + b2 * (u2 + v2);
    g[2] = w1 * (T(11) / T(6)) + w2 * (T(5) / T(6)) + w3 * (T(2) / T(6)) + b1 * (u1 + T(3) * v1) +
           b2 * (-T(2) * u2) + b3 * (u3 + T(3) * v3);
    g[3] = w2 * (T(2) / T(6)) + w3 * (T(5) / T(6)) + b2 * (u2 - v2) + b3 * (-T(2) * u3 - T(4) * v3);
    g[4] = w3 * (-T(1) / T(6)) + b3 * (u3 + v3);
    return h;
}

// Moments of one node (Eq. 10) in the form the derivatives use.
template <typename T>
struct Mom {
    T rho, ux, uy, E, Tm;
};
template <typename T>
__device__ __forceinline__ Mom<T> moments_of(const StepConst<T>& c, const T* f) {
    T r = 0, jx = 0, jy = 0, e = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        r += f[q];
        jx += f[q] * c.vx[q];
        jy += f[q] * c.vy[q];
        e += f[q] * c.v2[q];
    }
    Mom<T> m;
    const T ir = recip(r);
    m.rho = r;
    m.ux = jx * ir;
    m.uy = jy * ir;
    m.E = T(0.5) * e;
    m.Tm = m.E * ir - T(0.5) * (m.ux * m.ux + m.uy * m.uy);
    return m;
}

// G = sum_p lam_p d f^(0)_p / d(rho, u_x, u_y, T) at fixed (rho, u, T)
// (Eq. 28: f^(0) = rho F_k(T) B, B = A (1 + w) + w^2/2 + w^3/6, w = v.u/T,
// A = 1 - u^2/(2T)).
template <typename T>
__device__ __forceinline__ void feq_vjp_fields(const StepConst<T>& c, T rho, T ux, T uy, T Tm, const T* lam, T G[4]) {
    T F[4], dF[4];
    coeffs_and_slope(c, Tm, F, dF);
    const T u2 = ux * ux + uy * uy;
    const T iT = recip(Tm);  // the only reciprocal of the loop
    const T A = T(1) - T(0.5) * u2 * iT;
    T gr = 0, gx = 0, gy = 0, gT = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int k = ring_of(q);
        const T w = (c.vx[q] * ux + c.vy[q] * uy) * iT;
        const T B = A * (T(1) + w) + T(0.5) * w * w + w * w * w * (T(1) / T(6));
        const T dBw = A + w + T(0.5) * w * w;
        const T dBA = T(1) + w;
        const T lr = lam[q] * rho * F[k];
        gr += lam[q] * F[k] * B;
        gx += lr * (dBw * c.vx[q] - dBA * ux) * iT;
        gy += lr * (dBw * c.vy[q] - dBA * uy) * iT;
        gT += lam[q] * rho * dF[k] * B + lr * (-dBw * w + T(0.5) * dBA * u2 * iT) * iT;
    }
    G[0] = gr;
    G[1] = gx;
    G[2] = gy;
    G[3] = gT;
}

// the same sensitivity carried to the moments (rho, j_x, j_y, E):
// sum_p lam_p d f^(0)_p / d f_q = g[0] + g[1] v_qx + g[2] v_qy + g[3] |v_q|^2 / 2
template <typename T>
__device__ __forceinline__ void feq_vjp_moments(const StepConst<T>& c, const Mom<T>& m, const T* lam, T g[4]) {
    T G[4];
    feq_vjp_fields(c, m.rho, m.ux, m.uy, m.Tm, lam, G);
    const T ir = recip(m.rho);
    const T u2 = m.ux * m.ux + m.uy * m.uy;
    g[0] = G[0] - G[1] * m.ux * ir - G[2] * m.uy * ir + G[3] * (-m.E * ir * ir + u2 * ir);
    g[1] = (G[1] - G[3] * m.ux) * ir;
    g[2] = (G[2] - G[3] * m.uy) * ir;
    g[3] = G[3] * ir;
}

}  // namespace fdlb

namespace fdlb {

// ---------------------------------------------------------------------------
// kernels (one thread per face row position or per node)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T lam_at(const T* lam, const Geom& g, int q, int i, int j) {
    if (i < 0 || i >= g.nx || j < 0 || j >= g.ny) return T(0);  // ghosts are not state variables
    return lam[q * g.plane + (long long)(j + GY) * g.px + (i + GX)];
}

// the velocity of y slot k (the 12 velocities with v_y != 0: directions 1, 2,
// 4 and 5 of each ring) and the y slot of velocity q
__device__ __forceinline__ int yvel_of(int k) {
    const int d = k % 4;
    return 1 + 6 * (k / 4) + (d < 2 ? d : d + 1);
}
__device__ __forceinline__ int yslot_of(int q) {
    const int d = dir_of(q);
    return 4 * (ring_of(q) - 1) + (d < 3 ? d - 1 : d - 2);
}

// Face-gradient buffers, structure of arrays: entry k of the face at
// position t of velocity slot s lives at D[(5 s + k) nf + t].
// x faces: thread t = (i, j), i in [0, nx] the face between nodes i-1 and i
// of row j, for velocity q = blockIdx.y + 1 (every moving velocity has
// v_x != 0): the five entries mu * v * dh/dF.
template <typename T>
__device__ __forceinline__ void adj_faces_x(const StepConst<T>& c, const Geom& g, const T* __restrict__ f,
                                            const T* __restrict__ lam, T* __restrict__ D, int qx) {
    const long long nf = (long long)(g.nx + 1) * g.ny;
    const int q = qx + 1;
    const T v = c.vx[q];
    T* __restrict__ out = D + (long long)(5 * qx) * nf;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nf; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % (g.nx + 1)), j = (int)(t / (g.nx + 1));
        const T* row = f + q * g.plane + (long long)(j + GY) * g.px + GX;
        T a, b, cc, d, e;
        if (v > 0) {
            a = v * row[i - 3]; b = v * row[i - 2]; cc = v * row[i - 1]; d = v * row[i]; e = v * row[i + 1];
        } else {
            a = v * row[i + 2]; b = v * row[i + 1]; cc = v * row[i]; d = v * row[i - 1]; e = v * row[i - 2];
        }
        T gr[5];
        weno5_grad(a, b, cc, d, e, c.eps, gr);
        const T mu = c.dt / c.dx * (lam_at(lam, g, q, i, j) - lam_at(lam, g, q, i - 1, j)) * v;
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k * nf + t] = mu * gr[k];
    }
}

// y faces: thread t = (i, j), j in [0, ny] the face between rows j-1 and j of
// column i, for the velocity of y slot blockIdx.y
template <typename T>
__device__ __forceinline__ void adj_faces_y(const StepConst<T>& c, const Geom& g, const T* __restrict__ f,
                                            const T* __restrict__ lam, T* __restrict__ D, int qy) {
    const long long nf = (long long)g.nx * (g.ny + 1);
    const int q = yvel_of(qy);
    const T v = c.vy[q];
    T* __restrict__ out = D + (long long)(5 * qy) * nf;
    const long long P = g.px;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nf; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)(t / g.nx);
        const T* col = f + q * g.plane + (long long)GY * g.px + (i + GX);
        T a, b, cc, d, e;
        if (v > 0) {
            a = v * col[(j - 3) * P]; b = v * col[(j - 2) * P]; cc = v * col[(j - 1) * P];
            d = v * col[j * P]; e = v * col[(j + 1) * P];
        } else {
            a = v * col[(j + 2) * P]; b = v * col[(j + 1) * P]; cc = v * col[j * P];
            d = v * col[(j - 1) * P]; e = v * col[(j - 2) * P];
        }
        T gr[5];
        weno5_grad(a, b, cc, d, e, c.eps, gr);
        const T mu = c.dt / c.dy * (lam_at(lam, g, q, i, j) - lam_at(lam, g, q, i, j - 1)) * v;
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k * nf + t] = mu * gr[k];
    }
}

// Per node: the sensitivity of f^(0) carried to the moments (four values,
// feq_vjp_moments) and u_y (for the source term), into N[5][nx * ny].
template <typename T>
__device__ __forceinline__ void adj_node(const StepConst<T>& c, const Geom& g, const T* __restrict__ f,
                                         const T* __restrict__ lam, T* __restrict__ N) {
    const long long n = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)(t / g.nx);
        const long long at = (long long)(j + GY) * g.px + (i + GX);
        T fl[NQ], ll[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            fl[q] = f[q * g.plane + at];
            ll[q] = lam[q * g.plane + at];
        }
        const Mom<T> m = moments_of(c, fl);
        T gm[4];
        feq_vjp_moments(c, m, ll, gm);
#pragma unroll
        for (int k = 0; k < 4; ++k) N[k * n + t] = gm[k];
        N[4 * n + t] = m.uy;
    }
}

// Everything of a reverse step that reads only f^n and lambda^{n+1}, in one
// launch: blockIdx.y < 18 the x faces of velocity blockIdx.y + 1, 18 .. 29 the
// y faces of y slot blockIdx.y - 18, 30 the per-node moment sensitivities.
template <typename T>
__global__ void adj_faces_kernel(const StepConst<T> c, const Geom g, const T* __restrict__ f,
                                 const T* __restrict__ lam, T* __restrict__ Dx, T* __restrict__ Dy,
                                 T* __restrict__ N) {
    if (blockIdx.y < NQ - 1) adj_faces_x(c, g, f, lam, Dx, (int)blockIdx.y);
    else if (blockIdx.y < NQ - 1 + 12) adj_faces_y(c, g, f, lam, Dy, (int)blockIdx.y - (NQ - 1));
    else adj_node(c, g, f, lam, N);
}

// stencil positions that hold node i's value: the node itself and, next to a
// periodic or outflow side, its ghost images (a fixed-equilibrium ghost is a
// constant and carries no sensitivity)
__device__ __forceinline__ int images(int i, int n, int per, int lo_out, int hi_out, int pos[8]) {
    int m = 0;
    if (per) {
        for (int k = -3; k <= 3; ++k) {
            const int p = i + k * n;
            if (p >= -3 && p < n + 3) pos[m++] = p;
        }
        return m;
    }
    pos[m++] = i;
    if (i == 0 && lo_out) {
        pos[m++] = -1;
        pos[m++] = -2;
        pos[m++] = -3;
    }
    if (i == n - 1 && hi_out) {
        pos[m++] = n;
        pos[m++] = n + 1;
        pos[m++] = n + 2;
    }
    return m;
}

// lambda^n at interior node t = (i, j) for velocity q = blockIdx.y: the BGK
// adjoint, the gathered face entries and, with coef != 0, the source
// coef * dK/df of K = sum rho u_y^2 / 2.
template <typename T>
__global__ void adj_gather_kernel(const StepConst<T> c, const Geom g, const T* __restrict__ lam,
                                  const T* __restrict__ N, const T* __restrict__ Dx, const T* __restrict__ Dy,
                                  T coef, T* __restrict__ lam_out) {
    const long long n = (long long)g.nx * g.ny;
    const long long nfx = (long long)(g.nx + 1) * g.ny, nfy = (long long)g.nx * (g.ny + 1);
    const int q = blockIdx.y;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)(t / g.nx);
        const long long at = q * g.plane + (long long)(j + GY) * g.px + (i + GX);
        const T gm0 = N[t], gm1 = N[n + t], gm2 = N[2 * n + t], gm3 = N[3 * n + t];
        T acc = (T(1) - c.relax) * lam[at] +
                c.relax * (gm0 + gm1 * c.vx[q] + gm2 * c.vy[q] + gm3 * T(0.5) * c.v2[q]);
        if (coef != T(0)) {
            const T uy = N[4 * n + t];
            acc += coef * (uy * c.vy[q] - T(0.5) * uy * uy);
        }
        if (q > 0) {
            int pos_[8];
            const int np = images(i, g.nx, g.bcx_lo == 0, g.bcx_lo == 1, g.bcx_hi == 1, pos_);
            const T* Dq = Dx + (long long)(5 * (q - 1)) * nfx + (long long)j * (g.nx + 1);
            const bool pos = c.vx[q] > 0;
            for (int a = 0; a < np; ++a) {
                const int p = pos_[a];
                // faces i' whose stencil holds position p, and p's slot k in it
                const int lo = pos ? p - 1 : p - 2, hi = pos ? p + 3 : p + 2;
                for (int ip = (lo < 0 ? 0 : lo); ip <= (hi > g.nx ? g.nx : hi); ++ip) {
                    const int k = pos ? p - ip + 3 : ip + 2 - p;
                    acc += Dq[k * nfx + ip];
                }
            }
        }
        if (c.vy[q] != T(0)) {
            int pos_[8];
            const int np = images(j, g.ny, g.bcy_lo == 0, g.bcy_lo == 1, g.bcy_hi == 1, pos_);
            const T* Dq = Dy + (long long)(5 * yslot_of(q)) * nfy + i;
            const bool pos = c.vy[q] > 0;
            for (int a = 0; a < np; ++a) {
                const int p = pos_[a];
                const int lo = pos ? p - 1 : p - 2, hi = pos ? p + 3 : p + 2;
                for (int jp = (lo < 0 ? 0 : lo); jp <= (hi > g.ny ? g.ny : hi); ++jp) {
                    const int k = pos ? p - jp + 3 : jp + 2 - p;
                    acc += Dq[k * nfy + (long long)jp * g.nx];
                }
            }
        }
        lam_out[at] = acc;
    }
}

// lam = coef * dK/df (the sensitivity of the final state)
template <typename T>
__global__ void adj_source_kernel(const StepConst<T> c, const Geom g, const T* __restrict__ f, T coef,
                                  T* __restrict__ lam) {
    const long long n = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)(t / g.nx);
        const long long at = (long long)(j + GY) * g.px + (i + GX);
        T fl[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) fl[q] = f[q * g.plane + at];
        const Mom<T> m = moments_of(c, fl);
#pragma unroll
        for (int q = 0; q < NQ; ++q) lam[q * g.plane + at] = coef * (m.uy * c.vy[q] - T(0.5) * m.uy * m.uy);
    }
}

// dL/d(rho, u_x, u_y, T) of the initial fields from lambda^0 (f^0 = f^(0)(fields))
template <typename T>
__global__ void adj_fields_kernel(const StepConst<T> c, const Geom g, const double* __restrict__ rho,
                                  const double* __restrict__ ux, const double* __restrict__ uy,
                                  const double* __restrict__ Tm, const T* __restrict__ lam, double* __restrict__ d_rho,
                                  double* __restrict__ d_ux, double* __restrict__ d_uy, double* __restrict__ d_T) {
    const long long n = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)(t / g.nx);
        const long long at = (long long)(j + GY) * g.px + (i + GX);
        T ll[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) ll[q] = lam[q * g.plane + at];
        T G[4];
        feq_vjp_fields(c, T(rho[t]), T(ux[t]), T(uy[t]), T(Tm[t]), ll, G);
        d_rho[t] = G[0];
        d_ux[t] = G[1];
        d_uy[t] = G[2];
        d_T[t] = G[3];
    }
}

}  // namespace fdlb
