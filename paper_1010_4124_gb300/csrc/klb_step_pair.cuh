// klb_step_pair.cuh -- the fused FP32 step with two nodes per thread (tile
// variant 2): tiles of 32 columns x 16 rows, CTAs of 8 warps, warp w owning
// tile rows 2w and 2w + 1, two CTAs per SM.  Every per-node operation runs in
// packed f32x2 arithmetic across the two rows (lane x the upper row of the
// pair's first node, lane y the second), so one instruction serves two nodes
// where the one-node-per-thread variants spend one per node on the moments,
// F_k, f^(0), the conservative relaxation and the flux differences.  Each node
// gets exactly the operations, in the same order, that the other variants
// give it: the states are bitwise the same.
//
// Per tile (Eq. 47 of arXiv:1010.4124):
//  * the tile and its 3-node halo (all 19 planes) arrive by one TMA box load
//    (plain cp.async.bulk.tensor) into the CTA's single box buffer; the next
//    tile's load is issued as soon as every warp has read the box, and the
//    other CTA on the SM computes while a CTA waits for its load;
//  * x faces: the left face of each node for both rows as one packed WENO5
//    evaluation; the right face from lane L + 1 by shuffle, lane 31 from the
//    18 right-edge faces of the row pair evaluated up front;
//  * y faces: the faces below both rows as one packed evaluation; the upper
//    row's face below is the lower row's face above (a register), the face
//    above the upper row comes from the warp above through shared memory
//    (two face buffers in alternate tiles: one barrier per tile);
//  * diagnostics are not fused: a due sample is reduced by the stand-alone
//    kernel of the 32 x 16 tiles before the step.
#pragma once
#include "klb_pair.cuh"
#include "klb_step_f32.cuh"

namespace fdlb {

namespace v4 {
constexpr int TY = 16, NW = 8, NT = 32 * NW;
using S = v3::Shape<16>;                         // the box of a 32 x 16 tile (40 x 22 x 19 floats)
constexpr int YE = NW + 1;                       // face entries per y slot and column
constexpr int YF_FLOATS = v3::NYV * YE * 32;     // faces below the even rows 0, 2, .., 14 and above row 15
constexpr size_t SMEM_BYTES = sizeof(float) * (S::BUF_FLOATS + 2 * YF_FLOATS) + 128;
static_assert(v3::NYV / 2 <= NW, "one slot pair of top faces per warp");
}  // namespace v4

// the five upwind-ordered stencil values of the faces of rows r and r + 1 as
// pairs (x faces: left of column s; y faces: below each row)
template <int SGN>
__device__ __forceinline__ void xst2(const float* P, int r, int s, float2 v[5]) {
    float a[5], b[5];
    xst<SGN>(P, r, s, a);
    xst<SGN>(P, r + 1, s, b);
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = make_float2(a[k], b[k]);
}
template <int SGN>
__device__ __forceinline__ void yst2(const float* P, int r, int s, float2 v[5]) {
    float a[5], b[5];
    yst<SGN>(P, r, s, a);
    yst<SGN>(P, r + 1, s, b);
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = make_float2(a[k], b[k]);
}
__device__ __forceinline__ float2 weno_pair(const float2 v[5], float2 eps) {
    return ArithF32::weno2(v[0], v[1], v[2], v[3], v[4], eps);
}

// velocity Q with both components: x faces and the faces below of the pair
template <int Q>
__device__ __forceinline__ void pair_xy(const PairConst& pc, const float* tile, float* yf, int r, int s, int w,
                                        int lane, const float2* edge, float2* f) {
    constexpr int SGX = sgn_x(Q), SGY = sgn_y(Q);
    const float* P = tile + Q * v4::S::PLANE;
    float2 v[5];
    xst2<SGX>(P, r, s, v);
    const float2 hx = weno_pair(v, pc.ex[Q]);
    float2 hr = make_float2(__shfl_down_sync(0xffffffffu, hx.x, 1), __shfl_down_sync(0xffffffffu, hx.y, 1));
    if (lane == 31) hr = edge[Q - 1];  // the tile's right edge faces
    const float2 m1 = make_float2(-1.f, -1.f);
    f[Q] = __ffma2_rn(__fmul2_rn(pc.cx[Q], m1), __ffma2_rn(hx, m1, hr), f[Q]);
    yst2<SGY>(P, r, s, v);
    const float2 hy = weno_pair(v, pc.ey[Q]);
    f[Q] = __ffma2_rn(pc.cy[Q], hy, f[Q]);  // the faces below both nodes
    // the upper node's face above is the lower node's face below
    f[Q].x = fmaf(-pc.cy[Q].x, hy.y, f[Q].x);
    yf[(yslot(Q) * v4::YE + w) * 32 + lane] = hy.x;  // for the warp below: its lower node's face above
}
// velocity Q with an x component only
template <int Q>
__device__ __forceinline__ void pair_x(const PairConst& pc, const float* tile, int r, int s, int lane,
                                       const float2* edge, float2* f) {
    const float* P = tile + Q * v4::S::PLANE;
    float2 v[5];
    xst2<sgn_x(Q)>(P, r, s, v);
    const float2 hx = weno_pair(v, pc.ex[Q]);
    float2 hr = make_float2(__shfl_down_sync(0xffffffffu, hx.x, 1), __shfl_down_sync(0xffffffffu, hx.y, 1));
    if (lane == 31) hr = edge[Q - 1];
    const float2 m1 = make_float2(-1.f, -1.f);
    f[Q] = __ffma2_rn(__fmul2_rn(pc.cx[Q], m1), __ffma2_rn(hx, m1, hr), f[Q]);
}
// the faces above the tile's top row for y slots K and K + 1, lane's column
template <int K>
__device__ __forceinline__ void pair_top(const StepConst<float>& c, const float* tile, float* yf, int s, int lane) {
    constexpr int QA = yvel(K), QB = yvel(K + 1);
    float u[5], w[5];
    yst<sgn_y(QA)>(tile + QA * v4::S::PLANE, v4::TY + 3, s, u);
    yst<sgn_y(QB)>(tile + QB * v4::S::PLANE, v4::TY + 3, s, w);
    const float2 h = face_pair<0>(u, w, eps_pair(c, 22 + K / 2));
    yf[(K * v4::YE + v4::NW) * 32 + lane] = h.x;
    yf[((K + 1) * v4::YE + v4::NW) * 32 + lane] = h.y;
}
template <int K>
__device__ __forceinline__ void pair_tops(const StepConst<float>& c, const float* tile, float* yf, int s, int lane,
                                          int w) {
    if constexpr (K < v3::NYV) {
        if (w == K / 2) pair_top<K>(c, tile, yf, s, lane);
        pair_tops<K + 2>(c, tile, yf, s, lane, w);
    }
}

__global__ void __launch_bounds__(v4::NT, 2) step_pair_kernel(const __grid_constant__ StepConst<float> c,
                                                               const __grid_constant__ PairConst pc,
                                                               const InstDesc* __restrict__ desc, int ntiles,
                                                               int* __restrict__ err, long long spin_limit,
                                                               int inject) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* tile = reinterpret_cast<float*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    float* const yf0 = tile + v4::S::BUF_FLOATS;
    __shared__ __align__(8) uint64_t full;
    __shared__ __align__(8) uint64_t never;  // fault injection: a barrier nothing arrives on
    __shared__ float2 edges[v4::NW][v3::NXV];

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const Geom g = desc->g;
    float* const out = desc->out;
    const int tiles_x = desc->tiles_x;
    const float inv_tx = __frcp_rn((float)tiles_x);
    const uint32_t bar = smem_u32(&full);
    auto issue = [&](int t) {
        const TileInfo ti = tile_info<v4::TY>(t, tiles_x, inv_tx);
        tensormap_acquire(&desc->map);
        mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(float) * v4::S::BOX_FLOATS));
        tma_load_3d(smem_u32(tile), &desc->map, ti.bxa, ti.y0, 0, bar);
    };
    __syncthreads();
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(smem_u32(&never), 1);
        fence_barrier_init();
        fence_proxy_async();
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x);
    }
    __syncthreads();

    int k = 0;  // local tile counter: barrier phase and face buffer
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        bool late = !mbar_wait_bounded(bar, k & 1, spin_limit);
        if (inject) late = late || !mbar_wait_bounded(smem_u32(&never), 0, spin_limit);
        float* yf = yf0 + (k & 1) * v4::YF_FLOATS;
        const TileInfo ti = tile_info<v4::TY>(t, tiles_x, inv_tx);
        const int ix = ti.x0 + lane, iy = ti.y0 + 2 * w;
        const int s = lane + 4, r = 2 * w + 3;  // smem column of the nodes, smem row of the upper one
        const bool xin = ix >= 0 && ix < g.nx;
        const bool act0 = xin && iy < g.ny, act1 = xin && iy + 1 < g.ny;
        float2* const edge = edges[w];

        float2 f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            f[q] = make_float2(tile[q * v4::S::PLANE + r * v3::SXB + s], tile[q * v4::S::PLANE + (r + 1) * v3::SXB + s]);
        const NodeEq2 st = ArithF32x2::node_state(pc, f);
        ArithF32x2::collide(pc, st, f);  // f <- post-collision values
        // the right-edge x faces of both rows: lane j < 18 evaluates velocity j + 1
        if (lane < v3::NXV) {
            const int q = lane + 1;
            const bool pos = sgn_x(q) > 0;
            const int o = pos ? -3 : 2, d = pos ? 1 : -1;  // upwind stencil order (mirror for v_x < 0)
            const float* a = tile + q * v4::S::PLANE + r * v3::SXB + (v3::TW + 4);
            const float* b = a + v3::SXB;
            edge[lane] = ArithF32::weno2(make_float2(a[o], b[o]), make_float2(a[o + d], b[o + d]),
                                         make_float2(a[o + 2 * d], b[o + 2 * d]),
                                         make_float2(a[o + 3 * d], b[o + 3 * d]),
                                         make_float2(a[o + 4 * d], b[o + 4 * d]), pc.ex[q]);
        }
        __syncwarp();
        pair_xy<1>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<2>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<4>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<5>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<7>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<8>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<10>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<11>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<13>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<14>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<16>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_xy<17>(pc, tile, yf, r, s, w, lane, edge, f);
        pair_x<3>(pc, tile, r, s, lane, edge, f);
        pair_x<6>(pc, tile, r, s, lane, edge, f);
        pair_x<9>(pc, tile, r, s, lane, edge, f);
        pair_x<12>(pc, tile, r, s, lane, edge, f);
        pair_x<15>(pc, tile, r, s, lane, edge, f);
        pair_x<18>(pc, tile, r, s, lane, edge, f);
        pair_tops<0>(c, tile, yf, s, lane, w);
        // every face is in registers or in the face buffer: the box is free
        if (__syncthreads_or(late)) {
            if (tid == 0) {
                atomicOr(err, ERR_TIMEOUT);
                mbar_wait_bounded(bar, k & 1, kDrainPolls);  // let the copy land before leaving
            }
            __syncthreads();
            return;
        }
        if (tid == 0 && t + (int)gridDim.x < ntiles) {
            fence_proxy_async();
            issue(t + gridDim.x);
        }
        // the lower node's face above: the face below the next row pair
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            if (sgn_y(q) != 0) f[q].y = fmaf(-pc.cy[q].x, yf[(yslot(q) * v4::YE + w + 1) * 32 + lane], f[q].y);
        }
        const long long at = (long long)(iy + GY) * g.px + (ix + GX);
        if (act0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                KLB_GUARD(at + q * g.plane, NQ * g.plane) __stwb(out + at + q * g.plane, f[q].x);
            }
            if (has_images(g, ix, iy)) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) write_images(out, g, q, ix, iy, f[q].x);
            }
        }
        if (act1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                KLB_GUARD(at + g.px + q * g.plane, NQ * g.plane) __stwb(out + at + g.px + q * g.plane, f[q].y);
            }
            if (has_images(g, ix, iy + 1)) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) write_images(out, g, q, ix, iy + 1, f[q].y);
            }
        }
    }
}

}  // namespace fdlb
