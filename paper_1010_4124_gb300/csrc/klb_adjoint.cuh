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

// ---------------------------------------------------------------------------
// The reverse step in two launches.
//
// lambda^n_q(p) = (1 - dt/tau) lambda^{n+1}_q(p)
//               + dt/tau sum_r lambda^{n+1}_r(p) d f^(0)_r(p) / d f_q(p)      (BGK, Eq. 28)
//               + sum over the faces whose WENO5 stencil holds p of
//                 mu(face) dh(face)/dF at p, mu = dt/dx v (lambda(right) - lambda(left))
//               + the objective's source at sampled steps.
// A face's stencil may hold a ghost position, which is an image of an
// interior node (periodic wrap or outflow copy, Eqs. 57, 63-64): the tile
// kernel leaves those sums in the ghost cells of lambda^n, and the node
// kernel of the next reverse step (or the final fold) adds each ghost cell to
// the interior node it images and clears it.  So lambda's ghost cells are
// zero whenever a tile kernel reads them.
// ---------------------------------------------------------------------------

// Per interior node: fold the ghost-image sums of lambda into the node (and
// clear them); with NODE, also the f^(0) sensitivity carried to the moments
// (feq_vjp_moments, four values) and u_y into N[5][nx * ny].
template <typename T, bool NODE>
__global__ void adj_node_kernel(const StepConst<T> c, const Geom g, const T* __restrict__ f, T* __restrict__ lam,
                                T* __restrict__ N) {
    const long long n = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)(t / g.nx);
        const long long at = (long long)(j + GY) * g.px + (i + GX);
        int px_[8], py_[8];
        const int mx = images(i, g.nx, g.bcx_lo == 0, g.bcx_lo == 1, g.bcx_hi == 1, px_);
        const int my = images(j, g.ny, g.bcy_lo == 0, g.bcy_lo == 1, g.bcy_hi == 1, py_);
        T ll[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            T* L = lam + q * g.plane;
            T v = L[at];
            if (mx > 1 || my > 1) {
                for (int a = 0; a < mx; ++a)
                    if (px_[a] != i) {
                        T* cell = L + (long long)(j + GY) * g.px + (px_[a] + GX);
                        v += *cell;
                        *cell = T(0);
                    }
                for (int a = 0; a < my; ++a)
                    if (py_[a] != j) {
                        T* cell = L + (long long)(py_[a] + GY) * g.px + (i + GX);
                        v += *cell;
                        *cell = T(0);
                    }
                L[at] = v;
            }
            ll[q] = v;
        }
        if (NODE) {
            T fl[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) fl[q] = f[q * g.plane + at];
            const Mom<T> m = moments_of(c, fl);
            T gm[4];
            feq_vjp_moments(c, m, ll, gm);
#pragma unroll
            for (int k = 0; k < 4; ++k) N[k * n + t] = gm[k];
            N[4 * n + t] = m.uy;
        }
    }
}

// Tiles of the reverse step: 32 x TY positions of the extended grid (columns
// -4 .. nx + 2, rows -3 .. ny + 2: interior nodes and the ghost positions
// whose sums the node kernel folds back).  One CTA per (tile, velocity q).
template <int TY>
struct AdjTile {
    static constexpr int TX = 32;
    static __host__ __device__ int tiles_x(int nx) { return (nx + GX + 3 + TX - 1) / TX; }
    static __host__ __device__ int tiles_y(int ny) { return (ny + 2 * GY + TY - 1) / TY; }
};

// One CTA: velocity q = blockIdx.y on tile blockIdx.x.  f^n_q is staged with
// a halo of 5 positions (the stencils of the faces within 3 of the tile), and
// lambda^{n+1}_q with a halo of 3 (the faces' mu); every face whose stencil
// reaches the tile is evaluated once into shared memory (the 5 entries
// mu dh/dF), and each position gathers the entries that touch it.
template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY) adj_tile_kernel(const StepConst<T> c, const Geom g, const T* __restrict__ f,
                                                           const T* __restrict__ lam, const T* __restrict__ N, T coef,
                                                           T* __restrict__ lam_out) {
    constexpr int TX = AdjTile<TY>::TX;
    __shared__ T fs[TY + 10][TX + 10];  // positions (y0 - 5 + r, x0 - 5 + s)
    __shared__ T ls[TY + 6][TX + 6];    // positions (y0 - 3 + r, x0 - 3 + s)
    __shared__ T gx[5][TY][TX + 5];     // x face i = x0 - 2 + s of row y0 + r
    __shared__ T gy[5][TY + 5][TX];     // y face j = y0 - 2 + s of column x0 + l
    const int q = blockIdx.y;
    const int tiles_x = AdjTile<TY>::tiles_x(g.nx);
    const int x0 = (int)(blockIdx.x % tiles_x) * TX - GX;
    const int y0 = (int)(blockIdx.x / tiles_x) * TY - GY;
    const int tid = threadIdx.x, l = tid & 31, w = tid >> 5;
    const T* F = f + q * g.plane;
    const T* L = lam + q * g.plane;
    const T vx = c.vx[q], vy = c.vy[q];

    for (int k = tid; k < (TY + 10) * (TX + 10); k += 32 * TY) {
        const int r = k / (TX + 10), s = k - r * (TX + 10);
        const int y = y0 - 5 + r, x = x0 - 5 + s;
        const bool in = y >= -GY && y < g.ny + GY && x >= -GX && x < g.px - GX;
        fs[r][s] = in ? F[(long long)(y + GY) * g.px + (x + GX)] : T(0);
    }
    for (int k = tid; k < (TY + 6) * (TX + 6); k += 32 * TY) {
        const int r = k / (TX + 6), s = k - r * (TX + 6);
        const int y = y0 - 3 + r, x = x0 - 3 + s;
        const bool in = y >= 0 && y < g.ny && x >= 0 && x < g.nx;  // ghosts are not state variables
        ls[r][s] = in ? L[(long long)(y + GY) * g.px + (x + GX)] : T(0);
    }
    __syncthreads();
    if (q > 0) {
        const T cx = c.dt / c.dx;
        for (int k = tid; k < TY * (TX + 5); k += 32 * TY) {
            const int r = k / (TX + 5), s = k - r * (TX + 5);
            const int i = x0 - 2 + s, y = y0 + r;
            T gr[5] = {T(0), T(0), T(0), T(0), T(0)};
            T mu = T(0);
            if (i >= 0 && i <= g.nx && y >= 0 && y < g.ny) {
                const T* row = &fs[r + 5][0];
                if (vx > T(0))
                    weno5_grad(vx * row[s], vx * row[s + 1], vx * row[s + 2], vx * row[s + 3], vx * row[s + 4], c.eps,
                               gr);
                else
                    weno5_grad(vx * row[s + 5], vx * row[s + 4], vx * row[s + 3], vx * row[s + 2], vx * row[s + 1],
                               c.eps, gr);
                mu = cx * (ls[r + 3][s + 1] - ls[r + 3][s]) * vx;
            }
#pragma unroll
            for (int e = 0; e < 5; ++e) gx[e][r][s] = mu * gr[e];
        }
        if (vy != T(0)) {
            const T cy = c.dt / c.dy;
            for (int k = tid; k < (TY + 5) * TX; k += 32 * TY) {
                const int s = k / TX, ll = k - s * TX;
                const int j = y0 - 2 + s, x = x0 + ll;
                T gr[5] = {T(0), T(0), T(0), T(0), T(0)};
                T mu = T(0);
                if (j >= 0 && j <= g.ny && x >= 0 && x < g.nx) {
                    const int cl = ll + 5;
                    if (vy > T(0))
                        weno5_grad(vy * fs[s][cl], vy * fs[s + 1][cl], vy * fs[s + 2][cl], vy * fs[s + 3][cl],
                                   vy * fs[s + 4][cl], c.eps, gr);
                    else
                        weno5_grad(vy * fs[s + 5][cl], vy * fs[s + 4][cl], vy * fs[s + 3][cl], vy * fs[s + 2][cl],
                                   vy * fs[s + 1][cl], c.eps, gr);
                    mu = cy * (ls[s + 1][ll + 3] - ls[s][ll + 3]) * vy;
                }
#pragma unroll
                for (int e = 0; e < 5; ++e) gy[e][s][ll] = mu * gr[e];
            }
        }
    }
    __syncthreads();
    const int x = x0 + l, y = y0 + w;
    const bool xin = x >= 0 && x < g.nx, yin = y >= 0 && y < g.ny;
    const bool xg = (x >= -GX + 1 && x < 0) || (x >= g.nx && x < g.nx + 3);
    const bool yg = (y >= -GY && y < 0) || (y >= g.ny && y < g.ny + 3);
    if (!((xin && yin) || (xg && yin) || (xin && yg))) return;
    T acc = T(0);
    if (q > 0 && yin) {  // x faces whose stencil holds position x (its slot e in that stencil)
        if (vx > T(0)) {
#pragma unroll
            for (int e = 0; e < 5; ++e) acc += gx[e][w][l + 5 - e];
        } else {
#pragma unroll
            for (int e = 0; e < 5; ++e) acc += gx[e][w][l + e];
        }
    }
    if (q > 0 && vy != T(0) && xin) {
        if (vy > T(0)) {
#pragma unroll
            for (int e = 0; e < 5; ++e) acc += gy[e][w + 5 - e][l];
        } else {
#pragma unroll
            for (int e = 0; e < 5; ++e) acc += gy[e][w + e][l];
        }
    }
    const long long at = q * g.plane + (long long)(y + GY) * g.px + (x + GX);
    if (xin && yin) {
        const long long n = (long long)g.nx * g.ny, t = (long long)y * g.nx + x;
        const T gm0 = N[t], gm1 = N[n + t], gm2 = N[2 * n + t], gm3 = N[3 * n + t];
        T v = (T(1) - c.relax) * ls[w + 3][l + 3] + c.relax * (gm0 + gm1 * vx + gm2 * vy + gm3 * T(0.5) * c.v2[q]);
        if (coef != T(0)) {
            const T uy = N[4 * n + t];
            v += coef * (uy * vy - T(0.5) * uy * uy);
        }
        lam_out[at] = v + acc;
    } else {
        lam_out[at] = acc;  // a ghost position: its sum waits for the fold
    }
}

// lam := src[19][ny][nx] on the interior; the ghost cells stay zero (the
// fold of the reverse sweep reads them as pending image sums)
template <typename T>
__global__ void adj_import_kernel(const Geom g, const double* __restrict__ src, T* __restrict__ lam) {
    const long long n = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < NQ * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / n);
        const long long r = t - q * n;
        const int i = (int)(r % g.nx), j = (int)(r / g.nx);
        lam[q * g.plane + (long long)(j + GY) * g.px + (i + GX)] = T(src[t]);
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
