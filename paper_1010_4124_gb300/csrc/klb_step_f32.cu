// klb_step_f32.cu -- host side of the FP32 step (tile shapes, grid sizing,
// launch) and its WENO5 instances; the lower-order schemes are instanced in
// klb_step_f32_lo.cu.  The kernel itself is in klb_step_f32.cuh.
#include "klb_step_f32.cuh"

namespace fdlb {

static int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// tile heights offered: 16 rows (one CTA of 16 warps per SM) or 8 rows (two
// CTAs of 8 warps per SM, whose phases interleave)
static int rows_of(int variant) { return variant == 1 ? 8 : 16; }

void f32_tiles(int nx, int ny, int variant, int* tiles_x, int* ntiles) {
    const int ty = rows_of(variant);
    *tiles_x = (nx + GX + v3::TW - 1) / v3::TW;  // array columns 0 .. nx + GX - 1
    *ntiles = *tiles_x * ((ny + ty - 1) / ty);
}
int f32_grid(int nx, int ny, int variant) {
    int tx, nt;
    f32_tiles(nx, ny, variant, &tx, &nt);
    const int n = num_sms() * (16 / rows_of(variant));
    return nt < n ? nt : n;
}
// The faster tile shape by grid size, measured on GB300 (4096^2: 16-row tiles
// 15.1 vs 14.7 Gcell/s; 1024^2: 10.9 vs 11.7; 512^2: 5.9 vs 7.3): 8-row tiles
// (two CTAs per SM) up to 40 sixteen-row tiles per SM, 16-row tiles beyond.
int f32_default_variant(int nx, int ny) {
    int tiles_x, ntiles;
    f32_tiles(nx, ny, 0, &tiles_x, &ntiles);
    return ntiles <= 40 * num_sms() ? 1 : 0;
}
void f32_box(int variant, unsigned* bx, unsigned* by, unsigned* bz) {
    *bx = v3::SXB;
    *by = rows_of(variant) + 6;
    *bz = NQ;
}

cudaError_t prepare_f32_kernels() {
    num_sms();
    cudaError_t e = set_attr_f32<8, 0, false>();
    if (e == cudaSuccess) e = set_attr_f32<16, 0, false>();
    if (e == cudaSuccess) e = set_attr_f32<8, 0, true>();
    return e != cudaSuccess ? e : set_attr_f32<16, 0, true>();
}

cudaError_t launch_step_f32(const StepConst<float>& c, const InstDesc* descs, int ninst, int ntiles,
                            double* diag_partials, int* err, long long spin_limit, int inject, int variant,
                            cudaStream_t stream) {
    if (ninst < 1 || ninst > kMaxInstances) return cudaErrorInvalidValue;
    const int per_sm = 16 / rows_of(variant);
    const int grid = ntiles < num_sms() * per_sm ? ntiles : num_sms() * per_sm;
    if (grid < 1) return cudaSuccess;
    if (c.scheme != 0)
        return launch_step_f32_lo(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject,
                                  rows_of(variant), grid, stream);
    const bool multi = ninst > 1;
    if (rows_of(variant) == 8)
        return multi ? launch_f32_t<8, 0, true>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid,
                                                stream)
                     : launch_f32_t<8, 0, false>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject,
                                                 grid, stream);
    return multi ? launch_f32_t<16, 0, true>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid,
                                             stream)
                 : launch_f32_t<16, 0, false>(c, descs, ninst, ntiles, diag_partials, err, spin_limit, inject, grid,
                                              stream);
}

cudaError_t launch_diag_f32_batch(const StepConst<float>& c, const DiagJob* jobs, int njobs, int total_ctas,
                                  int variant, DueMask due, cudaStream_t s) {
    if (njobs < 1 || total_ctas < 1) return cudaSuccess;
    if (rows_of(variant) == 8)
        diag_f32_batch_kernel<8><<<total_ctas, 256, 0, s>>>(c, jobs, njobs, due);
    else
        diag_f32_batch_kernel<16><<<total_ctas, 512, 0, s>>>(c, jobs, njobs, due);
    return cudaGetLastError();
}

cudaError_t launch_diag_f32(const StepConst<float>& c, const Geom& g, const float* f, double* partials, int variant,
                            cudaStream_t s) {
    int tiles_x, ntiles;
    f32_tiles(g.nx, g.ny, variant, &tiles_x, &ntiles);
    const int grid = f32_grid(g.nx, g.ny, variant);
    if (rows_of(variant) == 8)
        diag_f32_kernel<8><<<grid, 256, 0, s>>>(c, g, tiles_x, ntiles, f, partials);
    else
        diag_f32_kernel<16><<<grid, 512, 0, s>>>(c, g, tiles_x, ntiles, f, partials);
    return cudaGetLastError();
}

KLB_BOUNDS_QUERY(bounds_flag_step_f32)

}  // namespace fdlb
