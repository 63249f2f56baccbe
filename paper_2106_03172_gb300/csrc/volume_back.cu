// Back projections for volumes (K2 + K3): slice stacks (nz independent
// slices sharing one 2-D geometry) and multi-ring scanners (fully 3-D lines
// of response through a voxel volume), each ending in the same per-pixel
// update as the single-slice kernels (epilogue.cuh).  The multi-ring weights
// come from the expressions the forward projector uses (piece_fraction /
// piece_zeta / layer_fraction), so A^T is the exact transpose of A.
#include "epilogue.cuh"

namespace petvr {

namespace {

// Slice-stack path: the geometry is shared by every slice.  A warp takes 4
// consecutive pixels and a window of 8 ZW consecutive slices; its lanes are
// 4 pixel groups x 8 z-lanes, and z-lane l carries slices l, l + 8, ... of the
// window, so each ratio load reads 8 consecutive floats of a bin's slice
// column ([view][bin][z]: coalesced).  The groups walk the subset's views in
// the same order (their candidate bins differ by about one, so the warp stays
// converged).  In each view, z-lane l of a group evaluates the band piece of
// candidate bin jlo + l of its pixel and the group's lanes take the weight by
// a shuffle; views and candidates are added in order (deterministic).  Each
// lane then applies the update to its own slices.
template <int EPI, typename TQ, bool GENPOT, int ZW>
__global__ void __launch_bounds__(kBlock) back_stack_kernel(const BackArgs a) {
    extern __shared__ unsigned char smem_raw[];
    ViewParams *s_views = reinterpret_cast<ViewParams *>(smem_raw);
    const int t = a.t_dev ? __ldg(a.t_dev) : a.t0 + (int)blockIdx.y;
    const int vb = __ldg(a.sub_off + t);
    const int nv = __ldg(a.sub_off + t + 1) - vb;
    int *s_vid = reinterpret_cast<int *>(s_views + nv);
    stage_views(a, vb, nv, s_views, s_vid);
    __syncthreads();
    const int r_view0 = a.t_dev ? vb : a.r_view0;

    // 32-bit index arithmetic: images and sinograms are below 2^31 elements (checked at plan time)
    const int n_win = (a.nz + 8 * ZW - 1) / (8 * ZW);
    const int lane = threadIdx.x & 31;
    const int zl = lane & 7;                              // z-lane
    const int pg = lane >> 3;                             // pixel group
    const unsigned gmask = 0xffu << (8 * pg);             // the group's 8 z-lanes
    const int wid = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    const int quad = wid / n_win;
    const int win = wid - quad * n_win;
    const int n = kStackPixels * quad + pg;               // pixel
    const bool live = n < a.nx * a.ny;
    const int ix = n % a.nx;
    const int iy = n / a.nx;
    const int z0 = win * 8 * ZW + zl;                     // this lane's first slice
    const int n_zi = live ? min(ZW, max(0, (a.nz - z0 + 7) / 8)) : 0;

    float acc[ZW];
#pragma unroll
    for (int i = 0; i < ZW; ++i) acc[i] = 0.0f;
    if (live) {
        for (int q = 0; q < nv; ++q) {
            const ViewParams vp = s_views[q];
            const int v = s_vid[q];
            const int k = vp.col ? ix : iy;              // major index
            const int minor = vp.col ? iy : ix;
            const int n_major = vp.col ? a.nx : a.ny;
            const int n_minor = vp.col ? a.ny : a.nx;
            const int mrel = minor - (n_minor >> 1);
            const float kc = (float)k - 0.5f * (float)n_major;
            int jlo, jhi;
            candidate_bins(vp, kc, (float)mrel, (float)mrel + 1.0f, a.nb, jlo, jhi);
            const float2 *ucv = a.uc + v * a.nb;
            const float *rv = a.r + (vb + q - r_view0) * a.nb * a.nz + z0;
            for (int jb = jlo; jb <= jhi; jb += 8) {     // the same trip count for the group's 8 lanes
                const int j = jb + zl;
                float w = 0.0f;
                if (j <= jhi) {
                    const float2 u = __ldg(ucv + j);
                    float fl, w0, w1;
                    band_split(vp, band_point(vp, u.y, kc), band_point(vp, u.y, kc + 1.0f), fl, w0, w1);
                    const int c0 = (int)fl + (int)u.x;
                    w = (c0 == mrel) ? w0 : ((c0 + 1 == mrel) ? w1 : 0.0f);
                }
                const int nc = min(8, jhi - jb + 1);
                for (int b = 0; b < nc; ++b) {
                    const float wb = __shfl_sync(gmask, w, b, 8);
                    if (wb == 0.0f) continue;
                    const float *rj = rv + (jb + b) * a.nz;
#pragma unroll
                    for (int i = 0; i < ZW; ++i)
                        if (i < n_zi) acc[i] = fmaf(wb, __ldg(rj + 8 * i), acc[i]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ZW; ++i)
        if (i < n_zi) {
            const int z = z0 + 8 * i;
            apply_epilogue<EPI, TQ, GENPOT>(a, t, (long long)n * a.nz + z, n, ix, iy, z, acc[i]);
        }
}

// Multi-ring path: kLanes lanes per voxel share the subset's views (lane l
// takes views l, l+4, ...).  For each candidate bin the band piece of the
// voxel's pixel is found as in the slice-stack path; each ring pair then adds
// the part of that piece inside the voxel's layer (piece_fraction /
// piece_zeta / layer_fraction, the forward projector's own expressions).
template <int EPI, typename TQ, bool GENPOT>
__global__ void __launch_bounds__(kBlock) ring_back_kernel(const BackArgs a) {
    extern __shared__ unsigned char smem_raw[];
    ViewParams *s_views = reinterpret_cast<ViewParams *>(smem_raw);
    const int t = a.t_dev ? __ldg(a.t_dev) : a.t0 + (int)blockIdx.y;
    const int vb = __ldg(a.sub_off + t);
    const int nv = __ldg(a.sub_off + t + 1) - vb;
    int *s_vid = reinterpret_cast<int *>(s_views + nv);
    stage_views(a, vb, nv, s_views, s_vid);
    __syncthreads();
    const int r_view0 = a.t_dev ? vb : a.r_view0;

    // 32-bit index arithmetic: images and sinograms are below 2^31 elements (checked at plan time)
    const int L = a.nz, P = a.pairs;
    const int plane = a.nx * a.ny * L;
    const long long gid = (long long)blockIdx.x * kBlock + threadIdx.x;
    const long long i = gid / kLanes;                    // voxel
    const int lane = (int)(gid % kLanes);
    const bool live = i < plane;
    const int iv = (int)i;
    const int iz = iv % L;
    const int n = iv / L;
    const int ix = n % a.nx;
    const int iy = n / a.nx;

    float acc = 0.0f;
    if (live) {
        for (int q = lane; q < nv; q += kLanes) {
            const ViewParams vp = s_views[q];
            const int v = s_vid[q];
            const int k = vp.col ? ix : iy;              // major index
            const int minor = vp.col ? iy : ix;
            const int n_major = vp.col ? a.nx : a.ny;
            const int n_minor = vp.col ? a.ny : a.nx;
            const int mrel = minor - (n_minor >> 1);
            const float kc = (float)k - 0.5f * (float)n_major;
            int jlo, jhi;
            candidate_bins(vp, kc, (float)mrel, (float)mrel + 1.0f, a.nb, jlo, jhi);
            const float2 *ucv = a.uc + v * a.nb;
            const float4 *lzv = a.lz + v * a.nb * P;
            const float *rv = a.r + (vb + q - r_view0) * a.nb * P;
            for (int j = jlo; j <= jhi; ++j) {
                const float2 u = __ldg(ucv + j);
                float fl, w0, w1;
                band_split(vp, band_point(vp, u.y, kc), band_point(vp, u.y, kc + 1.0f), fl, w0, w1);
                const int c0 = (int)fl + (int)u.x;
                const int side = (c0 == mrel) ? 0 : ((c0 + 1 == mrel && w1 > 0.0f) ? 1 : -1);
                if (side < 0) continue;
                const float w = side ? w1 : w0;
                float f_lo, f_hi;
                piece_fraction(vp, w0, w1, side == 1, f_lo, f_hi);
                for (int pr = 0; pr < P; ++pr) {
                    const float4 lz = __ldg(lzv + j * P + pr);
                    const float fr = layer_fraction(piece_zeta(lz, kc, f_lo), piece_zeta(lz, kc, f_hi), iz);
                    if (fr > 0.0f) acc = fmaf((w * lz.z) * fr, __ldg(rv + j * P + pr), acc);
                }
            }
        }
    }
#pragma unroll
    for (int o = kLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!live || lane != 0) return;
    apply_epilogue<EPI, TQ, GENPOT>(a, t, i, n, ix, iy, iz, acc);
}

// Multi-ring path for volumes of at most LMAX layers: kLanes lanes per pixel
// column share the subset's views; every candidate bin's band piece is found
// once per pixel and each ring pair's share is added to the layers its axial
// range crosses (per-layer sums in registers).  After the lane sum, lane l
// applies the update to layers l, l + kLanes, ..., one round at a time.
template <int EPI, typename TQ, bool GENPOT, int LMAX>
__global__ void __launch_bounds__(kBlock) ring_back_column_kernel(const BackArgs a) {
    extern __shared__ unsigned char smem_raw[];
    ViewParams *s_views = reinterpret_cast<ViewParams *>(smem_raw);
    const int t = a.t_dev ? __ldg(a.t_dev) : a.t0 + (int)blockIdx.y;
    const int vb = __ldg(a.sub_off + t);
    const int nv = __ldg(a.sub_off + t + 1) - vb;
    int *s_vid = reinterpret_cast<int *>(s_views + nv);
    stage_views(a, vb, nv, s_views, s_vid);
    __syncthreads();
    const int r_view0 = a.t_dev ? vb : a.r_view0;

    // 32-bit index arithmetic: images and sinograms are below 2^31 elements (checked at plan time)
    const int L = a.nz, P = a.pairs;
    const int npix = a.nx * a.ny;
    const int gid = blockIdx.x * kBlock + threadIdx.x;
    const int n = gid / kLanes;                          // pixel
    const int lane = gid % kLanes;
    const bool live = n < npix;
    const int ix = n % a.nx;
    const int iy = n / a.nx;

    float acc[LMAX];
#pragma unroll
    for (int iz = 0; iz < LMAX; ++iz) acc[iz] = 0.0f;
    if (live) {
        for (int q = lane; q < nv; q += kLanes) {
            const ViewParams vp = s_views[q];
            const int v = s_vid[q];
            const int k = vp.col ? ix : iy;              // major index
            const int minor = vp.col ? iy : ix;
            const int n_major = vp.col ? a.nx : a.ny;
            const int n_minor = vp.col ? a.ny : a.nx;
            const int mrel = minor - (n_minor >> 1);
            const float kc = (float)k - 0.5f * (float)n_major;
            int jlo, jhi;
            candidate_bins(vp, kc, (float)mrel, (float)mrel + 1.0f, a.nb, jlo, jhi);
            const float2 *ucv = a.uc + v * a.nb;
            const float4 *lzv = a.lz + v * a.nb * P;
            const float *rv = a.r + (vb + q - r_view0) * a.nb * P;
            for (int j = jlo; j <= jhi; ++j) {
                const float2 u = __ldg(ucv + j);
                float fl, w0, w1;
                band_split(vp, band_point(vp, u.y, kc), band_point(vp, u.y, kc + 1.0f), fl, w0, w1);
                const int c0 = (int)fl + (int)u.x;
                const int side = (c0 == mrel) ? 0 : ((c0 + 1 == mrel && w1 > 0.0f) ? 1 : -1);
                if (side < 0) continue;
                const float w = side ? w1 : w0;
                float f_lo, f_hi;
                piece_fraction(vp, w0, w1, side == 1, f_lo, f_hi);
                for (int pr = 0; pr < P; ++pr) {
                    const float4 lz = __ldg(lzv + j * P + pr);
                    const float za = piece_zeta(lz, kc, f_lo), zb = piece_zeta(lz, kc, f_hi);
                    const int il = (int)floorf(fminf(za, zb)), ih = (int)floorf(fmaxf(za, zb));
                    if (ih < 0 || il >= L) continue;
                    const float wr = __ldg(rv + j * P + pr);
#pragma unroll
                    for (int iz = 0; iz < LMAX; ++iz) {
                        if (iz < il || iz > ih || iz >= L) continue;
                        const float fr = layer_fraction(za, zb, iz);
                        if (fr > 0.0f) acc[iz] = fmaf((w * lz.z) * fr, wr, acc[iz]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int iz = 0; iz < LMAX; ++iz)
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) acc[iz] += __shfl_xor_sync(0xffffffffu, acc[iz], o);
    if (!live) return;
    // round e: lane l updates layer kLanes e + l, so the warp runs each
    // round's epilogue once
    static_assert(LMAX % kLanes == 0, "whole rounds of lanes");
#pragma unroll
    for (int e = 0; e < LMAX / kLanes; ++e) {
        float val = acc[e * kLanes];
#pragma unroll
        for (int l = 1; l < kLanes; ++l)
            if (lane == l) val = acc[e * kLanes + l];
        const int iz = e * kLanes + lane;
        if (iz < L) apply_epilogue<EPI, TQ, GENPOT>(a, t, n * L + iz, n, ix, iy, iz, val);
    }
}

// Back-projection launches of one epilogue / table type / potential.
struct VolumeBack {
    const BackArgs &a;
    int ny_grid;
    cudaStream_t s;
    int max_views;

    template <int EPI, typename TQ, bool GENPOT>
    pet_status run() const {
        const size_t smem = (size_t)max_views * (sizeof(ViewParams) + sizeof(int));
        if (a.axial && a.nz <= 8) {                     // multi-ring, layers in registers
            const int threads = a.nx * a.ny * kLanes;
            const dim3 grid((unsigned)((threads + kBlock - 1) / kBlock), (unsigned)ny_grid);
            if (a.nz <= 4)
                ring_back_column_kernel<EPI, TQ, GENPOT, 4><<<grid, kBlock, smem, s>>>(a);
            else
                ring_back_column_kernel<EPI, TQ, GENPOT, 8><<<grid, kBlock, smem, s>>>(a);
            return check_launch("ring_back_column_kernel");
        }
        if (a.axial) {                                  // multi-ring, one voxel per lane group
            const long long threads = (long long)a.nx * a.ny * a.nz * kLanes;
            const dim3 grid((unsigned)((threads + kBlock - 1) / kBlock), (unsigned)ny_grid);
            ring_back_kernel<EPI, TQ, GENPOT><<<grid, kBlock, smem, s>>>(a);
            return check_launch("ring_back_kernel");
        }
        // one warp per kStackPixels pixels and slice window
        const int zw = stack_lane_slices(a.nz);
        const long long quads = ((long long)a.nx * a.ny + kStackPixels - 1) / kStackPixels;
        const long long warps = quads * stack_windows(a.nz);
        const dim3 grid((unsigned)((warps + kBlock / 32 - 1) / (kBlock / 32)), (unsigned)ny_grid);
        switch (zw) {
            case 2: back_stack_kernel<EPI, TQ, GENPOT, 2><<<grid, kBlock, smem, s>>>(a); break;
            case 4: back_stack_kernel<EPI, TQ, GENPOT, 4><<<grid, kBlock, smem, s>>>(a); break;
            case 6: back_stack_kernel<EPI, TQ, GENPOT, 6><<<grid, kBlock, smem, s>>>(a); break;
            default: back_stack_kernel<EPI, TQ, GENPOT, 8><<<grid, kBlock, smem, s>>>(a); break;
        }
        return check_launch("back_stack_kernel");
    }
};

}  // namespace

pet_status launch_back_volume(const BackArgs &a, int epi, int table_dtype, int n_subsets_grid, cudaStream_t s,
                              int max_views) {
    return with_epilogue(epi, table_dtype, a.pot, VolumeBack{a, n_subsets_grid, s, max_views});
}

}  // namespace petvr
