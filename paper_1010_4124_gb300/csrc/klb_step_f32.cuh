// klb_step_f32.cuh -- the fused FDLB time step in FP32 (production path):
// device code, templated on the tile height and the convection scheme.
//
// One launch = one forward-Euler step (Eq. 47 of arXiv:1010.4124) over the
// whole grid.  Design, chosen so that every WENO5 face flux is evaluated
// once, occupancy stays high and barriers are few:
//
//  * Persistent CTAs (one per SM, 16 warps; or two of 8 warps) walk a list
//    of tiles of 32 columns x 16 (or 8) rows.  Warp w owns tile row w; lane
//    L owns array column 32 tx + L, so each warp-row store fills exactly one
//    128-byte line and neighbouring tiles never write into the same line.
//  * Each tile (all 19 planes plus a 3-node halo, 4 columns on the left so
//    the box starts on a 16-byte boundary) arrives by one 3-D TMA box load
//    (plain cp.async.bulk.tensor, no multicast) into one of two shared-memory
//    buffers; the load of the next tile is issued before the current one is
//    computed, so copies overlap computation.  Waits are bounded.
//  * x fluxes: lane L evaluates the face on the LEFT of its column; its right
//    face is lane L+1's left face, taken with one shuffle.  The 18 faces on
//    the right edge of the row are evaluated first, one per lane, and lane 31
//    takes its right faces from them.
//  * y fluxes: each thread evaluates the face BELOW its node and leaves it in
//    shared memory; the faces above the tile's top row are evaluated by six
//    warps (two velocities each, packed); after one barrier each node reads the face
//    above it from its upper neighbour.  That barrier is the only one per
//    tile with 16-row tiles (two face buffers, used by alternate tiles); the
//    8-row tiles (two CTAs per SM, one face buffer) add one at the tile's end.
//  * Per node: moments, F_k, f^(0) and the conservative BGK relaxation
//    (ArithF32::collide) in registers, the flux divergence, and a coalesced
//    store; nodes next to a periodic or outflow side also write their ghost
//    images.  Optionally the diagnostics of the input nodes are reduced per
//    CTA (FP32 node values, FP64 sums); the stand-alone kernel below
//    reproduces the same order.
#pragma once
#include "klb_device.cuh"
#include "klb_launch.h"

namespace fdlb {

namespace v3 {
// A tile row is one warp: lane L holds array column 32 tx + L (interior column
// 32 tx + L - GX), so every warp-row store covers one whole 128-byte line and
// no two tiles share a line.  The tile's first lanes fall on the left ghost
// columns for tx = 0 (inactive there).
constexpr int TW = 32;   // columns per tile (one warp row)
constexpr int SXB = 40;  // box width: array columns 32 tx - 4 .. 32 tx + 35 (halo of the 33 faces)
constexpr int NXV = 18;  // velocities with an x component (all but the rest velocity)
constexpr int NYV = 12;  // velocities with a y component
static_assert((sizeof(float) * SXB) % 16 == 0, "box rows of 16-byte multiples");
// tile of TW columns x TY rows (TY warps per CTA, 16 / TY CTAs per SM)
template <int TY>
struct Shape {
    static constexpr int NT = 32 * TY;
    static constexpr int SYB = TY + 6;  // box height
    static constexpr int PLANE = SXB * SYB;
    static constexpr int BOX_FLOATS = NQ * PLANE;
    static constexpr int BUF_FLOATS = (BOX_FLOATS + 31) / 32 * 32;  // 128-byte multiple (TMA destination)
    static constexpr int YF_FLOATS = NYV * (TY + 1) * 32;
    // face buffers: two (alternating tiles) when one CTA holds the SM, so that
    // no barrier is needed at the end of a tile; one when two CTAs share it
    static constexpr int YB = TY == 16 ? 2 : 1;
    static constexpr size_t SMEM_BYTES = sizeof(float) * (2 * BUF_FLOATS + YB * YF_FLOATS) + 128;
    static_assert((sizeof(float) * BUF_FLOATS) % 128 == 0, "TMA destination must stay 128-byte aligned");
};
}  // namespace v3

// index of velocity q among the 12 with a non-zero y component
__host__ __device__ constexpr int yslot(int q) {
    int n = 0;
    for (int k = 1; k < q; ++k) n += sgn_y(k) != 0 ? 1 : 0;
    return n;
}
// the velocity in y slot k
__host__ __device__ constexpr int yvel(int k) {
    int n = 0;
    for (int q = 1; q < NQ; ++q)
        if (sgn_y(q) != 0) {
            if (n == k) return q;
            ++n;
        }
    return -1;
}

// the five upwind-ordered stencil values of the x-face on the left of smem
// column s in row r of plane P
template <int SGN>
__device__ __forceinline__ void xst(const float* P, int r, int s, float v[5]) {  // (independent of TY)
    const float* a = P + r * v3::SXB + s;
    if (SGN > 0) {
        v[0] = a[-3]; v[1] = a[-2]; v[2] = a[-1]; v[3] = a[0]; v[4] = a[1];
    } else {
        v[0] = a[2]; v[1] = a[1]; v[2] = a[0]; v[3] = a[-1]; v[4] = a[-2];
    }
}
// ... of the y-face below smem row r (between rows r-1 and r) of column s
template <int SGN>
__device__ __forceinline__ void yst(const float* P, int r, int s, float v[5]) {
    const float* a = P + r * v3::SXB + s;
    constexpr int S = v3::SXB;
    if (SGN > 0) {
        v[0] = a[-3 * S]; v[1] = a[-2 * S]; v[2] = a[-S]; v[3] = a[0]; v[4] = a[S];
    } else {
        v[0] = a[2 * S]; v[1] = a[S]; v[2] = a[0]; v[3] = a[-S]; v[4] = a[-2 * S];
    }
}
// entry i of the epsilon pairs of the step constants, as one 8-byte load
__device__ __forceinline__ float2 eps_pair(const StepConst<float>& c, int i) {
    return *reinterpret_cast<const float2*>(c.epair[i]);
}

// The flux of the convection scheme SCH (0 WENO5, Eqs. 48-55; 1 first-order
// upwind; 2 second-order upwind; 3 second-order TVD) from five upwind-ordered
// stencil values of the unscaled plane, for two faces at once (packed) and
// for one face.  Every scheme is odd-homogeneous in the stencil, so the
// factor v of F = v f stays in the update constants as for WENO5.  The
// scalar form performs each lane's operations of the packed one.
template <int SCH>
__device__ __forceinline__ float2 face_pair(const float u[5], const float w[5], float2 e) {
    const float2 b = make_float2(u[1], w[1]), c = make_float2(u[2], w[2]), d = make_float2(u[3], w[3]);
    if constexpr (SCH == 0) {
        return ArithF32::weno2(make_float2(u[0], w[0]), b, c, d, make_float2(u[4], w[4]), e);
    } else if constexpr (SCH == 1) {
        return c;
    } else {
        const float2 m1 = make_float2(-1.f, -1.f), k05 = make_float2(0.5f, 0.5f);
        const float2 dl = __ffma2_rn(b, m1, c);
        if constexpr (SCH == 2) return __ffma2_rn(k05, dl, c);
        const float2 dr = __ffma2_rn(c, m1, d);
        return __ffma2_rn(k05, make_float2(minmod(dl.x, dr.x), minmod(dl.y, dr.y)), c);
    }
}
template <int SCH>
__device__ __forceinline__ float face_one(float a, float b, float c, float d, float e, float eps) {
    if constexpr (SCH == 0) {
        return ArithF32::weno(a, b, c, d, e, eps);
    } else if constexpr (SCH == 1) {
        return c;
    } else {
        const float dl = fmaf(b, -1.f, c);
        if constexpr (SCH == 2) return fmaf(0.5f, dl, c);
        return fmaf(0.5f, minmod(dl, fmaf(c, -1.f, d)), c);
    }
}

// The right-edge x-faces of a tile row (the left faces of array column
// 32 tx + 32, next tile's lane 0): lane j < 18 evaluates velocity j + 1 and
// leaves it in the warp's edge row; lane 31 takes its right faces from there.
template <int TY, int SCH>
__device__ __forceinline__ void edge_faces(const StepConst<float>& c, const float* tile, int r, int lane,
                                           float* edge) {
    if (lane < v3::NXV) {
        const int q = lane + 1;
        const bool pos = sgn_x(q) > 0;
        const int o = pos ? -3 : 2, d = pos ? 1 : -1;  // upwind stencil order (mirror for v_x < 0)
        const float* a = tile + q * v3::Shape<TY>::PLANE + r * v3::SXB + (v3::TW + 4);
        edge[lane] = face_one<SCH>(a[o], a[o + d], a[o + 2 * d], a[o + 3 * d], a[o + 4 * d], c.ex[q]);
    }
    __syncwarp();
}

// pass A for velocity Q with both components: its x-face and its y-face in
// one packed evaluation; x flux into post[Q], bottom y-face into shared memory
template <int TY, int SCH, int Q>
__device__ __forceinline__ void pass_a_xy(const StepConst<float>& c, const float* tile, float* yf, int r, int s,
                                          int ty, int lane, const float* edge, float* post) {
    constexpr int SGX = sgn_x(Q), SGY = sgn_y(Q);
    static_assert(SGX != 0 && SGY != 0, "velocity with two components");
    const float* P = tile + Q * v3::Shape<TY>::PLANE;
    float u[5], w[5];
    xst<SGX>(P, r, s, u);
    yst<SGY>(P, r, s, w);
    const float2 h = face_pair<SCH>(u, w, eps_pair(c, Q));
    float hr = __shfl_down_sync(0xffffffffu, h.x, 1);
    if (lane == 31) hr = edge[Q - 1];  // the tile's right edge face
    post[Q] = fmaf(-c.cx[Q], __fsub_rn(hr, h.x), post[Q]);
    post[Q] = fmaf(c.cy[Q], h.y, post[Q]);  // the face below enters now, the face above after the barrier
    yf[(yslot(Q) * (TY + 1) + ty) * 32 + lane] = h.y;
}
// pass A for two velocities QA, QB with an x component only
template <int TY, int SCH, int QA, int QB>
__device__ __forceinline__ void pass_a_xx(const StepConst<float>& c, const float* tile, int r, int s, int lane,
                                          const float* edge, float* post) {
    static_assert(sgn_y(QA) == 0 && sgn_y(QB) == 0, "x-only velocities");
    float u[5], w[5];
    xst<sgn_x(QA)>(tile + QA * v3::Shape<TY>::PLANE, r, s, u);
    xst<sgn_x(QB)>(tile + QB * v3::Shape<TY>::PLANE, r, s, w);
    static_assert(QB == QA + 3 && (QA - 3) % 6 == 0, "x-only pairs (6m + 3, 6m + 6)");
    const float2 h = face_pair<SCH>(u, w, eps_pair(c, 19 + (QA - 3) / 6));
    float ra = __shfl_down_sync(0xffffffffu, h.x, 1);
    float rb = __shfl_down_sync(0xffffffffu, h.y, 1);
    if (lane == 31) {  // the tile's right edge faces
        ra = edge[QA - 1];
        rb = edge[QB - 1];
    }
    post[QA] = fmaf(-c.cx[QA], __fsub_rn(ra, h.x), post[QA]);
    post[QB] = fmaf(-c.cx[QB], __fsub_rn(rb, h.y), post[QB]);
}

// the faces above the tile's top row, velocities of y slots K and K + 1 (one
// packed evaluation), for lane's column
template <int TY, int SCH, int K>
__device__ __forceinline__ void top_face_pair(const StepConst<float>& c, const float* tile, float* yf, int s,
                                              int lane) {
    constexpr int QA = yvel(K), QB = yvel(K + 1);
    float u[5], w[5];
    yst<sgn_y(QA)>(tile + QA * v3::Shape<TY>::PLANE, TY + 3, s, u);
    yst<sgn_y(QB)>(tile + QB * v3::Shape<TY>::PLANE, TY + 3, s, w);
    const float2 h = face_pair<SCH>(u, w, eps_pair(c, 22 + K / 2));
    yf[(K * (TY + 1) + TY) * 32 + lane] = h.x;
    yf[((K + 1) * (TY + 1) + TY) * 32 + lane] = h.y;
}
// warp w < 6 evaluates the top faces of y slots 2w and 2w + 1
template <int TY, int SCH, int K>
__device__ __forceinline__ void top_faces(const StepConst<float>& c, const float* tile, float* yf, int s, int lane,
                                          int w) {
    static_assert(v3::NYV % 2 == 0 && v3::NYV / 2 <= TY, "one slot pair per warp");
    if constexpr (K < v3::NYV) {
        if (w == K / 2) top_face_pair<TY, SCH, K>(c, tile, yf, s, lane);
        top_faces<TY, SCH, K + 2>(c, tile, yf, s, lane, w);
    }
}

struct TileInfo {
    int x0, y0, bxa;
};
// t / d and t % d for 0 <= t < 2^24 and d >= 1, without an integer division:
// the quotient estimated from the correctly rounded reciprocal inv_d of d,
// corrected by one step (exact over that range)
__device__ __forceinline__ int2 tile_divmod(int t, int d, float inv_d) {
    int q = __float2int_rz(__fmul_rn(__int2float_rn(t), inv_d));
    int r = t - q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
    return make_int2(q, r);
}
template <int TY>
__device__ __forceinline__ TileInfo tile_info(int t, int tiles_x, float inv_tx) {
    TileInfo ti;
    const int2 qr = tile_divmod(t, tiles_x, inv_tx);
    const int tx = qr.y;
    ti.x0 = v3::TW * tx - GX;  // interior column of lane 0
    ti.y0 = qr.x * TY;
    ti.bxa = v3::TW * tx - 4;  // array column of the box start (16-byte aligned; -4 reads zeros)
    return ti;
}

// Tiles of several instances (grids of one batch, or the single grid of a
// handle) form one index space: instance i owns tiles [first_i, first_i + n_i).
// The CTA keeps the first-tile table in shared memory and finds a tile's
// instance by binary search.
__device__ __forceinline__ int find_inst(const int* first, int ninst, int t) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// acquire a tensor map that the host wrote to global memory before the launch
__device__ __forceinline__ void tensormap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// MULTI: the launch may cover several grids (a batch); a single grid
// (MULTI false) skips the instance lookup altogether.
template <int TY, int SCH, bool MULTI>
__global__ void __launch_bounds__(32 * TY, 16 / TY) step_f32_kernel(const __grid_constant__ StepConst<float> c,
                                                                    const InstDesc* __restrict__ descs, int ninst,
                                                                    int ntiles, double* __restrict__ diag_partials,
                                                                    int* __restrict__ err, long long spin_limit,
                                                                    int inject) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the launch reserves 128 spare bytes so that the buffers start on a
    // 128-byte boundary of the shared window whatever precedes them
    float* buf = reinterpret_cast<float*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    using S = v3::Shape<TY>;
    float* const yf0 = buf + 2 * S::BUF_FLOATS;
    __shared__ __align__(8) uint64_t full[2];
    __shared__ __align__(8) uint64_t never;  // fault injection: a barrier nothing arrives on
    __shared__ int first[kMaxInstances];
    // the instance of the tile in each buffer, written by the thread that
    // issues the copy and read by all after the next CTA barrier
    __shared__ int tile_inst[2];
    __shared__ float edges[TY][v3::NXV];

    const int tid = threadIdx.x, ty = tid >> 5, lane = tid & 31;
    for (int i = tid; i < ninst; i += blockDim.x) first[i] = descs[i].first_tile;
    auto issue = [&](int t, int b) {
        const int inst = MULTI ? find_inst(first, ninst, t) : 0;
        if (MULTI) tile_inst[b] = inst;
        const InstDesc* D = descs + inst;
        const TileInfo ti = tile_info<TY>(t - D->first_tile, D->tiles_x, __frcp_rn((float)D->tiles_x));
        const uint32_t bar = smem_u32(&full[b]);
        tensormap_acquire(&D->map);
        mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(float) * S::BOX_FLOATS));
        tma_load_3d(smem_u32(buf + b * S::BUF_FLOATS), &D->map, ti.bxa, ti.y0, 0, bar);
    };
    __syncthreads();
    if (tid == 0) {
        mbar_init(smem_u32(&full[0]), 1);
        mbar_init(smem_u32(&full[1]), 1);
        mbar_init(smem_u32(&never), 1);
        fence_barrier_init();
        fence_proxy_async();
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    }
    __syncthreads();

    DiagAccF32 acc;
    const bool diag = diag_partials != nullptr;
    // fields of the instance of the current tile, read from global memory
    // only when the instance changes (tiles of one instance are contiguous)
    int cur = -1, first_t = 0, tiles_x = 1;
    float inv_tx = 1.f;
    Geom g{};
    float* out = nullptr;
    int k = 0;  // local tile counter: buffer k & 1, phase (k >> 1) & 1
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        // prefetch the next tile into the other buffer (last read before the
        // middle barrier of the previous tile)
        if (tid == 0 && t + (int)gridDim.x < ntiles) {
            fence_proxy_async();
            issue(t + gridDim.x, b ^ 1);
        }
        // A wait that gives up is reported at the barrier in the middle of
        // the tile; until then the thread computes on whatever the buffer
        // holds (shared-memory reads only) and stores nothing.
        bool late = !mbar_wait_bounded(smem_u32(&full[b]), (k >> 1) & 1, spin_limit);
        if (inject) late = late || !mbar_wait_bounded(smem_u32(&never), 0, spin_limit);
        float* yf = yf0 + (S::YB == 2 ? b : 0) * S::YF_FLOATS;
        const int inst = MULTI ? tile_inst[b] : 0;
        if (inst != cur) {
            const InstDesc* D = descs + inst;
            g = D->g;
            out = D->out;
            first_t = D->first_tile;
            tiles_x = D->tiles_x;
            inv_tx = __frcp_rn((float)tiles_x);
            cur = inst;
        }
        const float* tile = buf + b * S::BUF_FLOATS;
        const TileInfo ti = tile_info<TY>(t - first_t, tiles_x, inv_tx);
        const int ix = ti.x0 + lane, iy = ti.y0 + ty;
        const int s = lane + 4;  // smem column of the node
        const int r = ty + 3;    // smem row of the node
        const bool active = ix >= 0 && ix < g.nx && iy < g.ny;
        float* const edge = edges[ty];

        float f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) f[q] = tile[q * S::PLANE + r * v3::SXB + s];
        const NodeEq<float> st = ArithF32::node_state(c, f);
        if (diag) acc.add(st, active);
        ArithF32::collide(c, st, f);  // f <- post-collision values
        edge_faces<TY, SCH>(c, tile, r, lane, edge);
        // x and y faces of the 12 velocities with two components, packed in pairs
        pass_a_xy<TY, SCH, 1>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 2>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 4>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 5>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 7>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 8>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 10>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 11>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 13>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 14>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 16>(c, tile, yf, r, s, ty, lane, edge, f);
        pass_a_xy<TY, SCH, 17>(c, tile, yf, r, s, ty, lane, edge, f);
        // x faces of the six velocities along the x axis, in pairs
        pass_a_xx<TY, SCH, 3, 6>(c, tile, r, s, lane, edge, f);
        pass_a_xx<TY, SCH, 9, 12>(c, tile, r, s, lane, edge, f);
        pass_a_xx<TY, SCH, 15, 18>(c, tile, r, s, lane, edge, f);
        top_faces<TY, SCH, 0>(c, tile, yf, s, lane, ty);  // faces above the tile's top row
        // All faces are in shared memory and nobody reads this tile buffer
        // again (the next copy into it is issued after this barrier).
        if (__syncthreads_or(late)) {
            if (tid == 0) {
                atomicOr(err, ERR_TIMEOUT);
                // let both copies that may be in flight land before leaving
                mbar_wait_bounded(smem_u32(&full[b]), (k >> 1) & 1, kDrainPolls);
                if (t + (int)gridDim.x < ntiles)
                    mbar_wait_bounded(smem_u32(&full[b ^ 1]), ((k + 1) >> 1) & 1, kDrainPolls);
            }
            __syncthreads();
            return;
        }
        // y fluxes: the face above each node (its upper neighbour's lower face)
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            if (sgn_y(q) != 0) f[q] = fmaf(-c.cy[q], yf[(yslot(q) * (TY + 1) + ty + 1) * 32 + lane], f[q]);
        }
        if (active) {
            const long long at = (long long)(iy + GY) * g.px + (ix + GX);
            float* o = out + at;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                KLB_GUARD(at + q * g.plane, NQ * g.plane) __stwb(o + q * g.plane, f[q]);  // global store
            }
            if (has_images(g, ix, iy)) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) write_images(out, g, q, ix, iy, f[q]);
            }
        }
        // With two face buffers, the next tile writes the other one, and the
        // one read here is written again only after every thread has passed
        // the next tile's middle barrier.  With one, wait for all readers.
        if (S::YB == 1) __syncthreads();
    }
    if (diag) diag_block_reduce<S::NT>(acc, diag_partials + 8ll * blockIdx.x);
}

// Diagnostics of a state with the same tiles, per-CTA tile order and block
// reduction as the fused path inside the step kernel, so that both give the
// same bits: CTA `cta` of `ncta` takes tiles cta, cta + ncta, ... and writes
// one partial record.
template <int TY>
__device__ __forceinline__ void diag_cta(const StepConst<float>& c, const Geom& g, int tiles_x, int ntiles,
                                         const float* __restrict__ f, double* __restrict__ partial, int cta,
                                         int ncta) {
    const int tid = threadIdx.x, ty = tid >> 5, lane = tid & 31;
    const float inv_tx = __frcp_rn((float)tiles_x);
    // the node of tile t for this thread, its activity and its 19 values
    auto load = [&](int t, float fl[NQ]) {
        const TileInfo ti = tile_info<TY>(t, tiles_x, inv_tx);
        const int ix = ti.x0 + lane, iy = ti.y0 + ty;
        const bool active = ix >= 0 && ix < g.nx && iy < g.ny;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            fl[q] = active ? KLB_LOAD(f, q * g.plane + (long long)(iy + GY) * g.px + (ix + GX), NQ * g.plane, 1.f) : 1.f;
        return active;
    };
    DiagAccF32 acc;
    // the loads of the next tile are issued before the current one is reduced
    // (two tiles in flight per thread); the accumulation order is unchanged
    float cur[NQ], nxt[NQ];
    bool act = cta < ntiles ? load(cta, cur) : false;
    for (int t = cta; t < ntiles; t += ncta) {
        const bool act_n = t + ncta < ntiles ? load(t + ncta, nxt) : false;
        acc.add(ArithF32::node_state(c, cur), act);
#pragma unroll
        for (int q = 0; q < NQ; ++q) cur[q] = nxt[q];
        act = act_n;
    }
    diag_block_reduce<32 * TY>(acc, partial);
}

template <int TY>
__global__ void __launch_bounds__(32 * TY) diag_f32_kernel(const StepConst<float> c, const Geom g, int tiles_x,
                                                           int ntiles, const float* __restrict__ f,
                                                           double* __restrict__ partials) {
    diag_cta<TY>(c, g, tiles_x, ntiles, f, partials + 8ll * blockIdx.x, blockIdx.x, gridDim.x);
}

// The stand-alone reductions of several members in one launch: CTA b belongs
// to the job whose CTA range holds b, and does that job's CTA b - first_cta.
template <int TY>
__global__ void __launch_bounds__(32 * TY) diag_f32_batch_kernel(const StepConst<float> c,
                                                                 const DiagJob* __restrict__ jobs, int njobs,
                                                                 const DueMask due) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first_cta <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    if (!KLB_DUE_BIT(due, lo)) return;  // uniform across the CTA
    const DiagJob& J = jobs[lo];
    const int v = (int)blockIdx.x - J.first_cta;
    diag_cta<TY>(c, J.g, J.tiles_x, J.ntiles, J.f, J.partials + 8ll * v, v, J.grid);
}

// dynamic shared memory of the kernel instance, set once per process
template <int TY, int SCH, bool MULTI>
cudaError_t set_attr_f32() {
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(step_f32_kernel<TY, SCH, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)v3::Shape<TY>::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

template <int TY, int SCH, bool MULTI>
cudaError_t launch_f32_t(const StepConst<float>& c, const InstDesc* descs, int ninst, int ntiles,
                         double* diag_partials, int* err, long long spin_limit, int inject, int grid,
                         cudaStream_t stream) {
    cudaError_t e = set_attr_f32<TY, SCH, MULTI>();
    if (e != cudaSuccess) return e;
    step_f32_kernel<TY, SCH, MULTI><<<grid, 32 * TY, v3::Shape<TY>::SMEM_BYTES, stream>>>(c, descs, ninst, ntiles,
                                                                                 diag_partials, err, spin_limit,
                                                                                 inject);
    return cudaGetLastError();
}

}  // namespace fdlb
