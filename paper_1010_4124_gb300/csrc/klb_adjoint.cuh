// klb_adjoint.cuh -- adjoint (vector-Jacobian product) of the FDLB step.
//
// For the step f^{n+1} = S(f^n) of Eq. (47) (arXiv:1010.4124) and a
// sensitivity lambda^{n+1} = dL/df^{n+1}, these kernels form
//   lambda^n = (dS/df^n)^T lambda^{n+1}
// on the interior nodes, with every dependence through ghost nodes folded back
// onto the interior node the ghost copies (periodic wrap, outflow copy).
// A reverse step is three launches:
//   * fold: the ghost-image sums the previous reverse step left in lambda's
//     ghost cells are added to the nodes they image;
//   * node: per node, the adjoint of the BGK term's f^(0) part,
//     (dt/tau) (d f^(0)/df)^T lambda, carried through the four moments
//     (rho, rho u, E) that f^(0) depends on;
//   * tile: per tile and velocity, every WENO5 face h (Eqs. 48-55 applied to
//     F = v f) whose stencil reaches the tile, its sensitivity
//     mu = dL/dh = (dt/dx)(lambda(right node) - lambda(left node)) times the
//     gradient of h with respect to its five stencil values, nonlinear weights
//     included, kept in shared memory; each node then gathers the entries of
//     the faces whose stencils contain it, plus (1 - dt/tau) lambda and the
//     node term; ghost positions keep their sums for the next fold.
// Sources and the initial state: dK/df for K = sum rho u_y^2 / 2, and
// (d f^(0) / d(rho, u_x, u_y, T))^T lambda^0 for the initial fields.
#pragma once
#include "klb_device.cuh"
#include "klb_launch.h"

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
// five inputs, in the difference form the FP32 step evaluates (its
// derivation is in ArithF32::weno): with D1 = a - b, D2 = c - b, D3 = d - c,
// E4 = d - e, the 3/4-scaled indicators s_q (eps34 = 3/4 eps), w_q = 1/s_q^2,
// G1 = 5/6 D2 + 1/3 D1, G2 = D2 + 2 D3, G3 = 2 D3 + E4/2 and the weights
// delta' = (1, 6, 3) (the optimal weights times 10),
//   h = c + N / D,  N = sum G_q w_q,  D = sum delta'_q w_q,
//   dh = dc + (1/D) [sum w_q dG_q + sum (G_q - delta'_q (h - c)) dw_q],
//   dw_q = -2 w_q / s_q ds_q.
// The partials with respect to (D1, D2, D3, E4) are mapped back to (a..e).
template <typename T>
__device__ __forceinline__ T weno5_grad(T a, T b, T c, T d, T e, T eps34, T g[5]) {
    const T D1 = a - b, D2 = c - b, D3 = d - c, E4 = d - e;
    const T s1 = D1 * (D1 + T(2.75) * D2) + T(2.5) * D2 * D2 + eps34;
    const T s2 = D2 * (D2 - T(1.25) * D3) + D3 * D3 + eps34;
    const T s3 = E4 * (E4 + T(2.75) * D3) + T(2.5) * D3 * D3 + eps34;
    const T r1 = recip(s1), r2 = recip(s2), r3 = recip(s3);
    const T w1 = r1 * r1, w2 = r2 * r2, w3 = r3 * r3;
    const T G1 = T(5.0 / 6.0) * D2 + T(1.0 / 3.0) * D1, G2 = D2 + T(2) * D3, G3 = T(2) * D3 + T(0.5) * E4;
    const T rD = recip(w1 + T(6) * w2 + T(3) * w3);
    const T hh = (G1 * w1 + G2 * w2 + G3 * w3) * rD;  // h - c
    const T o1 = w1 * rD, o2 = w2 * rD, o3 = w3 * rD;
    const T m = T(-2) * rD;
    const T b1 = m * (G1 - hh) * w1 * r1, b2 = m * (G2 - T(6) * hh) * w2 * r2, b3 = m * (G3 - T(3) * hh) * w3 * r3;
    const T g1 = T(1.0 / 3.0) * o1 + b1 * (T(2) * D1 + T(2.75) * D2);
    const T g2 = T(5.0 / 6.0) * o1 + o2 + b1 * (T(2.75) * D1 + T(5) * D2) + b2 * (T(2) * D2 - T(1.25) * D3);
    const T g3 = T(2) * (o2 + o3) + b2 * (T(2) * D3 - T(1.25) * D2) + b3 * (T(2.75) * E4 + T(5) * D3);
    const T g4 = T(0.5) * o3 + b3 * (T(2) * E4 + T(2.75) * D3);
    g[0] = g1;
    g[1] = -g1 - g2;
    g[2] = T(1) + g2 - g3;
    g[3] = g3 + g4;
    g[4] = -g4;
    return c + hh;
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
// The reverse step in three launches.
//
// lambda^n_q(p) = (1 - dt/tau) lambda^{n+1}_q(p)
//               + dt/tau sum_r lambda^{n+1}_r(p) d f^(0)_r(p) / d f_q(p)      (BGK, Eq. 28)
//               + sum over the faces whose WENO5 stencil holds p of
//                 mu(face) dh(face)/dF at p, mu = dt/dx v (lambda(right) - lambda(left))
//               + the objective's source at sampled steps.
// A face's stencil may hold a ghost position, which is an image of an
// interior node (periodic wrap or outflow copy, Eqs. 57, 63-64): the tile
// kernel leaves those sums in the ghost cells of lambda^n, and the fold
// kernel of the next reverse step (or after the last one) adds each ghost
// cell to the interior node it images and clears it.  So lambda's ghost
// cells are zero whenever a tile kernel reads them.
// ---------------------------------------------------------------------------

// Ghost cells that image interior node (i, j): along x (cells of the same
// row) and along y (of the same column).  Periodic: ghost p images node p mod
// n; outflow: the three ghosts beyond an edge node image it (the adjoint is
// not offered for fixed-equilibrium sides).  Up to 6 + 6 cells (grids
// narrower than 3 nodes wrap several times); offsets into one plane.
__device__ __forceinline__ int image_cells(const Geom& g, int i, int j, long long cell[12]) {
    int m = 0;
    const long long row = (long long)(j + GY) * g.px;
    if (g.bcx_lo == 0) {
        for (int k = -3; k <= 3; ++k) {
            const int p = i + k * g.nx;
            if (k != 0 && ((p >= -3 && p < 0) || (p >= g.nx && p < g.nx + 3))) cell[m++] = row + p + GX;
        }
    } else {
        if (i == 0 && g.bcx_lo == 1)
            for (int d = 1; d <= 3; ++d) cell[m++] = row + GX - d;
        if (i == g.nx - 1 && g.bcx_hi == 1)
            for (int d = 0; d < 3; ++d) cell[m++] = row + g.nx + GX + d;
    }
    if (g.bcy_lo == 0) {
        for (int k = -3; k <= 3; ++k) {
            const int p = j + k * g.ny;
            if (k != 0 && ((p >= -3 && p < 0) || (p >= g.ny && p < g.ny + 3)))
                cell[m++] = (long long)(p + GY) * g.px + i + GX;
        }
    } else {
        if (j == 0 && g.bcy_lo == 1)
            for (int d = 1; d <= 3; ++d) cell[m++] = (long long)(GY - d) * g.px + i + GX;
        if (j == g.ny - 1 && g.bcy_hi == 1)
            for (int d = 0; d < 3; ++d) cell[m++] = (long long)(g.ny + GY + d) * g.px + i + GX;
    }
    return m;
}

// The columns (rows) whose nodes have x (y) images: the band next to a
// periodic pair of sides (all of them on grids of at most 6), or the edge
// nodes of outflow sides.  band_count gives their number, band_at the k-th.
__host__ __device__ __forceinline__ int band_count(int n, int lo, int hi) {
    if (lo == 0) return n < 6 ? n : 6;
    return n == 1 ? ((lo == 1 || hi == 1) ? 1 : 0) : (lo == 1) + (hi == 1);
}
__host__ __device__ __forceinline__ int band_at(int n, int lo, int hi, int k) {
    if (lo == 0) return n <= 6 ? k : (k < 3 ? k : n - 6 + k);
    return (k == 0 && lo == 1) ? 0 : n - 1;
}

// Fold the ghost-image sums of lambda into the nodes they image (and clear
// the ghost cells).  One thread per (node with images, velocity): first the
// nodes of the x band (their y images too), then those of the y band that
// have no x images.  All loads of a thread precede its stores.
template <typename T>
__global__ void adj_fold_kernel(const Geom g, T* __restrict__ lam, int nbx, int nby) {
    const int nxb = nbx * g.ny, nyb = nby * g.nx, per_q = nxb + nyb;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < NQ * per_q; t += gridDim.x * blockDim.x) {
        const int q = t / per_q, r = t - q * per_q;
        int i, j;
        if (r < nxb) {
            j = r / nbx;
            i = band_at(g.nx, g.bcx_lo, g.bcx_hi, r - j * nbx);
        } else {
            const int r2 = r - nxb;
            const int k = r2 / g.nx;
            i = r2 - k * g.nx;
            j = band_at(g.ny, g.bcy_lo, g.bcy_hi, k);
            const bool xe = g.bcx_lo == 0 ? (i < 3 || i >= g.nx - 3)
                                          : ((i == 0 && g.bcx_lo == 1) || (i == g.nx - 1 && g.bcx_hi == 1));
            if (xe) continue;  // folded with the x band
        }
        T* L = lam + q * g.plane;
        long long cell[12];
        const int m = image_cells(g, i, j, cell);
        const long long at = (long long)(j + GY) * g.px + (i + GX);
        const long long lim = (NQ - q) * g.plane;  // the cells of planes q .. 18 from L
        (void)lim;  // read by the guards of the bounds-checked build only
        T v = KLB_LOAD(L, at, lim, T(0));
        for (int k = 0; k < m; ++k) v += KLB_LOAD(L, cell[k], lim, T(0));
        for (int k = 0; k < m; ++k) {
            KLB_GUARD(cell[k], lim) L[cell[k]] = T(0);
        }
        KLB_GUARD(at, lim) L[at] = v;
    }
}

// Per interior node, on a folded lambda: the f^(0) sensitivity carried to
// the moments (feq_vjp_moments, four values) and u_y into N[5][nx * ny].  One
// CTA per segment of kNodeSeg nodes of row j = blockIdx.y: the segment's 19
// planes of f and of lambda arrive by two TMA box loads (kNodeSeg x 1 x 19)
// on a bounded mbarrier, so all 38 values of a node are fetched at once.
constexpr int kNodeSeg = 128;
template <typename T>
__global__ void __launch_bounds__(kNodeSeg) adj_node_kernel(const __grid_constant__ CUtensorMap fmap,
                                                            const __grid_constant__ CUtensorMap lmap,
                                                            const StepConst<T> c, const Geom g, T* __restrict__ N,
                                                            int* __restrict__ err, long long spin_limit) {
    __shared__ __align__(128) T fsm[NQ][kNodeSeg];
    __shared__ __align__(128) T lsm[NQ][kNodeSeg];
    __shared__ __align__(8) uint64_t bar;
    const int j = blockIdx.y, i0 = blockIdx.x * kNodeSeg, tid = threadIdx.x;
    const uint32_t b = smem_u32(&bar);
    if (tid == 0) {
        mbar_init(b, 1);
        fence_barrier_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(b, (uint32_t)(2 * sizeof(T) * NQ * kNodeSeg));
        tma_load_3d(smem_u32(&fsm[0][0]), &fmap, i0 + GX, j + GY, 0, b);
        tma_load_3d(smem_u32(&lsm[0][0]), &lmap, i0 + GX, j + GY, 0, b);
    }
    __syncthreads();
    const bool late = !mbar_wait_bounded(b, 0, spin_limit);
    if (__syncthreads_or(late)) {
        if (tid == 0) {
            atomicOr(err, ERR_TIMEOUT);
            mbar_wait_bounded(b, 0, kDrainPolls);  // let the copies land before the CTA leaves
        }
        __syncthreads();
        return;
    }
    const int i = i0 + tid;
    if (i >= g.nx) return;
    T ll[NQ], fl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        ll[q] = lsm[q][tid];
        fl[q] = fsm[q][tid];
    }
    const Mom<T> m = moments_of(c, fl);
    T gm[4];
    feq_vjp_moments(c, m, ll, gm);
    const long long n = (long long)g.nx * g.ny, t = (long long)j * g.nx + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        KLB_GUARD(k * n + t, 5 * n) N[k * n + t] = gm[k];
    }
    KLB_GUARD(4 * n + t, 5 * n) N[4 * n + t] = m.uy;
}

// Tiles of the reverse step: 32 x TY interior positions (tile (bx, by) starts
// at node (32 bx, TY by)).  One CTA per (tile, velocity q).  Both staged boxes
// are BW = 48 positions wide and start 8 positions left of the tile's lane 0
// (array column 32 bx - 4: 16-byte aligned for TMA): the f box holds rows
// -5 .. TY + 4 of the tile, the lambda box rows -3 .. TY + 2.  The ghost
// positions next to the grid's edges (whose sums the fold kernel adds back)
// are gathered by the tiles at those edges, from faces they hold anyway.
template <typename T, int TY>
struct AdjTile {
    static constexpr int TX = 32, BW = 48;
    static constexpr int FR = TY + 10, LR = TY + 6;
    static __host__ __device__ int tiles_x(int nx) { return (nx + TX - 1) / TX; }
    static __host__ __device__ int tiles_y(int ny) { return (ny + TY - 1) / TY; }
    static_assert((BW * sizeof(T)) % 16 == 0, "TMA box rows of 16-byte multiples");
    static_assert((FR * BW * sizeof(T)) % 128 == 0 && (LR * BW * sizeof(T)) % 128 == 0, "boxes keep 128-byte alignment");
};

// The faces and the gather of one CTA for a velocity whose components have
// the signs SX, SY (compile time, so no branch on them remains): every face
// whose stencil reaches the tile is evaluated once into shared memory (the
// five entries mu dh/dF), and each position gathers the entries that touch
// it.  A face outside the grid (i < 0 or i > nx, or a row outside it) has
// mu = 0 since lambda is zero off the interior, so no face needs a validity
// test.  Threads map to faces in three fixed passes: x faces 0..31 of each
// row, y faces 0..TY-1 of each column, then the remaining 5 y-face rows
// (warps 0..4) and 5 x-face columns (warps 5.., 4 rows of 5 per warp).
template <typename T, int TY, int SX, int SY>
__device__ __forceinline__ void adj_tile_body(const StepConst<T>& c, const Geom& g, int q, int x0, int y0,
                                              const T (*fs)[AdjTile<T, TY>::BW], const T (*ls)[AdjTile<T, TY>::BW],
                                              T (*gx)[TY][AdjTile<T, TY>::TX + 5], T (*gy)[TY + 5][AdjTile<T, TY>::TX],
                                              const T* __restrict__ N, T coef, T* __restrict__ lam_out) {
    constexpr int TX = AdjTile<T, TY>::TX;
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    const T vx = c.vx[q], vy = c.vy[q], e34 = T(0.75) * c.eps;
    // box columns: f position x0 - 8 + col, lambda the same; face s of a row
    // lies between positions x0 - 3 + s and x0 - 2 + s (face i = x0 - 2 + s)
    auto face_x = [&](int r, int s) {
        const T* row = fs[r + 5];
        T gr[5];
        if (SX > 0)
            weno5_grad(vx * row[s + 3], vx * row[s + 4], vx * row[s + 5], vx * row[s + 6], vx * row[s + 7], e34, gr);
        else
            weno5_grad(vx * row[s + 8], vx * row[s + 7], vx * row[s + 6], vx * row[s + 5], vx * row[s + 4], e34, gr);
        const T mu = c.cx[q] * (ls[r + 3][s + 6] - ls[r + 3][s + 5]);  // dt v_x / dx times the jump of lambda
#pragma unroll
        for (int e = 0; e < 5; ++e) gx[e][r][s] = mu * gr[e];
    };
    // y face s of column cl: between rows y0 - 3 + s and y0 - 2 + s
    auto face_y = [&](int s, int cl) {
        const int x = cl + 8;
        T gr[5];
        if (SY > 0)
            weno5_grad(vy * fs[s][x], vy * fs[s + 1][x], vy * fs[s + 2][x], vy * fs[s + 3][x], vy * fs[s + 4][x], e34,
                       gr);
        else
            weno5_grad(vy * fs[s + 5][x], vy * fs[s + 4][x], vy * fs[s + 3][x], vy * fs[s + 2][x], vy * fs[s + 1][x],
                       e34, gr);
        const T mu = c.cy[q] * (ls[s + 1][x] - ls[s][x]);
#pragma unroll
        for (int e = 0; e < 5; ++e) gy[e][s][cl] = mu * gr[e];
    };
    if (SX != 0) {
        face_x(w, l);
        if (SY != 0) face_y(w, l);
        if (w < 5) {
            if (SY != 0) face_y(TY + w, l);
        } else if (l < 20) {
            const int rr = 4 * (w - 5) + l / 5;
            if (rr < TY) face_x(rr, TX + l % 5);
        }
    }
    __syncthreads();
    // ghost positions beyond the tile's own columns or rows at the grid's
    // edges: the 3 columns left of column 0 (and right of the last tile, past
    // its lanes) in the tile's rows, the 3 rows below row 0 (and above the last
    // tile row) in its columns; each sums the face entries whose slot falls
    // inside the tile's face arrays (the others belong to faces off the grid)
    {
        // the last tile column (row) takes the ghost columns (rows) past its lanes
        const int xr_lo = x0 == 0 ? 3 : 0;
        const int xr_hi = x0 + TX >= g.nx ? max(0, g.nx + 3 - (x0 + TX)) : 0;
        const int yr_lo = y0 == 0 ? 3 : 0;
        const int yr_hi = y0 + TY >= g.ny ? max(0, g.ny + 3 - (y0 + TY)) : 0;
        int k = threadIdx.x;
        const int nxr = (xr_lo + xr_hi) * TY;
        if (k < nxr) {  // an x rim position: column p, row y0 + r
            const int r = k / (xr_lo + xr_hi), m = k - r * (xr_lo + xr_hi);
            const int p = m < xr_lo ? m - 3 : x0 + TX + (m - xr_lo);
            const int y = y0 + r;
            if (SX != 0 && y < g.ny) {
                T acc = T(0);
#pragma unroll
                for (int e = 0; e < 5; ++e) {
                    const int sl = SX > 0 ? p - x0 + 5 - e : p - x0 + e;
                    if (sl >= 0 && sl < TX + 5) acc += gx[e][r][sl];
                }
                const long long at = q * g.plane + (long long)(y + GY) * g.px + (p + GX);
                KLB_GUARD(at, NQ * g.plane) lam_out[at] = acc;
            }
        } else if ((k -= nxr) < (yr_lo + yr_hi) * TX) {  // a y rim position: row p, column x0 + l
            const int r = k / TX, cl = k - r * TX;
            const int p = r < yr_lo ? r - 3 : y0 + TY + (r - yr_lo);
            const int x = x0 + cl;
            if (x < g.nx) {
                T acc = T(0);
                if (SY != 0) {
#pragma unroll
                    for (int e = 0; e < 5; ++e) {
                        const int sl = SY > 0 ? p - y0 + 5 - e : p - y0 + e;
                        if (sl >= 0 && sl < TY + 5) acc += gy[e][sl][cl];
                    }
                }
                const long long at = q * g.plane + (long long)(p + GY) * g.px + (x + GX);
                KLB_GUARD(at, NQ * g.plane) lam_out[at] = acc;
            }
        }
    }
    const int x = x0 + l, y = y0 + w;
    const bool xin = x >= 0 && x < g.nx, yin = y >= 0 && y < g.ny;
    const bool xg = (x >= -GX + 1 && x < 0) || (x >= g.nx && x < g.nx + 3);
    const bool yg = (y >= -GY && y < 0) || (y >= g.ny && y < g.ny + 3);
    if (!((xin && yin) || (xg && yin) || (xin && yg))) return;
    T acc = T(0);
    if (SX != 0 && yin) {  // x faces whose stencil holds position x (its slot e in that stencil)
#pragma unroll
        for (int e = 0; e < 5; ++e) acc += gx[e][w][SX > 0 ? l + 5 - e : l + e];
    }
    if (SY != 0 && xin) {
#pragma unroll
        for (int e = 0; e < 5; ++e) acc += gy[e][SY > 0 ? w + 5 - e : w + e][l];
    }
    const long long at = q * g.plane + (long long)(y + GY) * g.px + (x + GX);
    if (xin && yin) {
        const long long n = (long long)g.nx * g.ny, t = (long long)y * g.nx + x;
        const T gm0 = KLB_LOAD(N, t, 5 * n, T(0)), gm1 = KLB_LOAD(N, n + t, 5 * n, T(0));
        const T gm2 = KLB_LOAD(N, 2 * n + t, 5 * n, T(0)), gm3 = KLB_LOAD(N, 3 * n + t, 5 * n, T(0));
        T v = (T(1) - c.relax) * ls[w + 3][l + 8] + c.relax * (gm0 + gm1 * vx + gm2 * vy + gm3 * T(0.5) * c.v2[q]);
        if (coef != T(0)) {
            const T uy = KLB_LOAD(N, 4 * n + t, 5 * n, T(0));
            v += coef * (uy * vy - T(0.5) * uy * uy);
        }
        KLB_GUARD(at, NQ * g.plane) lam_out[at] = v + acc;
    } else {
        KLB_GUARD(at, NQ * g.plane) lam_out[at] = acc;  // a ghost position: its sum waits for the fold
    }
}

// One CTA: velocity q = blockIdx.y on tile blockIdx.x, reverse step nstep.  f^n_q (halo 5: the
// stencils of the faces within 3 of the tile) and lambda^{n+1}_q (halo 3: the
// faces' mu) arrive by two TMA box loads (plain cp.async.bulk.tensor, no
// multicast) on one mbarrier; a wait that runs out sets ERR_TIMEOUT.
// lambda's cells off the interior are zero (ghosts cleared by the fold, pads
// and corners never written), so the box needs no masking.
template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY) adj_tile_kernel(const __grid_constant__ CUtensorMap fmap,
                                                           const __grid_constant__ CUtensorMap lmap,
                                                           const StepConst<T> c, const Geom g,
                                                           const T* __restrict__ N, const double* __restrict__ coefs,
                                                           int nstep, T* __restrict__ lam_out, int* __restrict__ err,
                                                           long long spin_limit) {
    using A = AdjTile<T, TY>;
    constexpr int TX = A::TX;
    static_assert(TY >= 7, "the remainder pass needs warps 0..4 and two more");
    __shared__ __align__(128) T fs[A::FR][A::BW];
    __shared__ __align__(128) T ls[A::LR][A::BW];
    __shared__ T gx[5][TY][TX + 5];  // x face i = x0 - 2 + s of row y0 + r
    __shared__ T gy[5][TY + 5][TX];  // y face j = y0 - 2 + s of column x0 + l
    __shared__ __align__(8) uint64_t bar;
    const int q = blockIdx.y;
    const int tiles_x = A::tiles_x(g.nx);
    const int by = (int)blockIdx.x / tiles_x, bx = (int)blockIdx.x - by * tiles_x;
    const int x0 = bx * TX, y0 = by * TY;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_barrier_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(b, (uint32_t)(sizeof(T) * A::BW * (A::FR + A::LR)));
        // box origins (array coordinates): column x0 - 8 + GX, rows y0 - 5 + GY and y0 - 3 + GY
        tma_load_3d(smem_u32(&fs[0][0]), &fmap, x0 - 8 + GX, y0 - 5 + GY, q, b);
        tma_load_3d(smem_u32(&ls[0][0]), &lmap, x0 - 8 + GX, y0 - 3 + GY, q, b);
    }
    __syncthreads();
    const bool late = !mbar_wait_bounded(b, 0, spin_limit);
    if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) {
            atomicOr(err, ERR_TIMEOUT);
            mbar_wait_bounded(b, 0, kDrainPolls);  // let the copies land before the CTA leaves
        }
        __syncthreads();
        return;
    }
    const int sx = sgn_x(q), sy = sgn_y(q);  // uniform across the CTA
    // the objective's weight at this step (0 where no sample enters), read from
    // device memory so that a captured sweep serves every objective
    const T coef = T(coefs[nstep]);
#define KLB_ADJ_BODY(SX, SY) adj_tile_body<T, TY, SX, SY>(c, g, q, x0, y0, fs, ls, gx, gy, N, coef, lam_out)
    if (sx == 0) KLB_ADJ_BODY(0, 0);
    else if (sx > 0 && sy > 0) KLB_ADJ_BODY(1, 1);
    else if (sx > 0 && sy < 0) KLB_ADJ_BODY(1, -1);
    else if (sx > 0) KLB_ADJ_BODY(1, 0);
    else if (sy > 0) KLB_ADJ_BODY(-1, 1);
    else if (sy < 0) KLB_ADJ_BODY(-1, -1);
    else KLB_ADJ_BODY(-1, 0);
#undef KLB_ADJ_BODY
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
        const long long at = q * g.plane + (long long)(j + GY) * g.px + (i + GX);
        KLB_GUARD(at, NQ * g.plane) lam[at] = T(KLB_LOAD(src, t, NQ * n, 0.0));
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
        for (int q = 0; q < NQ; ++q) fl[q] = KLB_LOAD(f, q * g.plane + at, NQ * g.plane, T(0));
        const Mom<T> m = moments_of(c, fl);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            KLB_GUARD(q * g.plane + at, NQ * g.plane) lam[q * g.plane + at] = coef * (m.uy * c.vy[q] - T(0.5) * m.uy * m.uy);
        }
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
        for (int q = 0; q < NQ; ++q) ll[q] = KLB_LOAD(lam, q * g.plane + at, NQ * g.plane, T(0));
        T G[4];
        feq_vjp_fields(c, T(rho[t]), T(ux[t]), T(uy[t]), T(Tm[t]), ll, G);
        d_rho[t] = G[0];
        d_ux[t] = G[1];
        d_uy[t] = G[2];
        d_T[t] = G[3];
    }
}

}  // namespace fdlb
