// Forward projection with the Poisson-ratio epilogue (K1).
//
// yhat_m = sum_n a_mn f_n + w_m for the rays m of a view range (§2.1,
// Eq. (voxel_td)); in ratio mode the kernel writes r_m = g_m / yhat_m (the
// ratio inside every E-step and gradient, §2.2 Eq. (EMsurrogate), §2.3
// Eq. (tau_t), §4 Eq. (osem_additive)), 0 when yhat_m = 0 (§2.3 remedy), and
// optionally reduces the log-likelihood sum_m g_m log yhat_m - yhat_m (§2.1,
// Eq. (log_likelihood)) in FP64 to one partial per block.
//
// Thread layout: consecutive lanes share one ray, each walking a contiguous
// chunk of the ray's major bands, then an xor-shuffle all-reduce combines
// the chunks in a fixed order (deterministic).  Slice stacks (nz > 1) and
// multi-ring lines have their own kernels in volume.cu (a warp of band chunks
// x z-lanes per ray; the axial split of each piece).
//
// The view range is either given on the host (v_begin/v_end) or, when
// a.t_dev is set, read on the device from the subset offsets, so that one
// captured launch serves any subset; the grid then covers the largest subset
// and surplus threads only take part in the reduction.
#include <algorithm>

#include "bodies.cuh"

namespace petvr {

namespace {

// The kernels run beside the other streams' kernels: at 40 registers six
// blocks fit on an SM (five for the full-data ratio pass, which spills at 40).
template <int CHUNKS, bool LL>
constexpr int fwd_min_blocks() { return CHUNKS >= 32 || LL ? 6 : 5; }

template <int CHUNKS, int MODE, bool LL>
__global__ void __launch_bounds__(kBlock, fwd_min_blocks<CHUNKS, LL>()) forward_tile_kernel(const FwdArgs a) {
    forward_tile_body<CHUNKS, MODE, LL>(a, blockIdx.x);
}

// Persistent batched forward: a resident grid whose blocks claim work items
// (WorkSeg lists) until the list is exhausted.  An item is one block of the
// single-state forward launch of that member and kind, run by the same body
// with the same band-chunk count, so every ratio (and every log-likelihood
// block partial) is bit-identical to the member's own launches.  Thread 0
// claims the item and writes its arguments to shared memory (the body reads
// them there, as the single launch reads its kernel parameters); the segment
// table is staged in shared memory once per block.  The body's shared arrays
// are free again once the next claim's barrier has passed.
template <int MODE, bool LL>
__global__ void __launch_bounds__(kBlock, 6)
    persistent_forward_kernel(const BatchMember *ms, const WorkSeg *segs, int n_segs, int n_items, int iter,
                              int in_is_img, int *claim) {
    __shared__ WorkSeg s_segs[kSegSmem];
    __shared__ FwdArgs s_a;
    __shared__ int s_item, s_bx, s_shape;
    for (int i = threadIdx.x; i < n_segs && i < kSegSmem; i += blockDim.x) s_segs[i] = segs[i];
    const WorkSeg *tab = n_segs <= kSegSmem ? s_segs : segs;
    // the segment table and member descriptors were copied in before the
    // kernel ahead of this one; the claim counter was zeroed by a kernel, so
    // wait for the kernel ahead before the first claim
    pdl_wait();
    pdl_trigger();
    // the first item of each block is its own index; later ones are claimed
    // (the counter counts claims beyond the grid's first items)
    for (int round = 0;; ++round) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int g = round == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(claim, 1);
            s_item = g;
            if (g < n_items) {
                const WorkSeg sg = tab[find_segment(tab, n_segs, g)];
                const BatchMember &m = ms[sg.member];
                FwdArgs a{};
                a.views = m.views;
                a.uc = m.uc;
                a.order = m.order;
                a.nx = m.nx;
                a.ny = m.ny;
                a.nz = 1;
                a.nb = m.nb;
                a.g = m.g;
                a.w = m.w;
                a.w_scalar = m.w_scalar;
                a.status = m.status;
                if (sg.kind == WK_FWD_UPDATE) {
                    a.sub_off = m.sub_off;
                    a.t_dev = m.seq + iter;
                    a.img = in_is_img ? m.img : m.alt;
                    a.out = m.ratio;
                } else if (sg.kind == WK_FWD_ANCHOR) {
                    a.v_begin = 0;
                    a.v_end = m.na;
                    a.img = in_is_img ? m.img : m.alt;
                    a.out = m.ratio_full;
                } else {
                    a.v_begin = 0;
                    a.v_end = m.na;
                    a.img = m.img;
                    a.ll_partials = m.part;
                }
                s_a = a;
                s_bx = g - sg.first;
                s_shape = sg.shape;
            }
        }
        __syncthreads();
        if (s_item >= n_items) break;
        const int bx = s_bx;
        if (s_shape == 8)
            forward_tile_body<8, MODE, LL>(s_a, bx);
        else if (s_shape == 16)
            forward_tile_body<16, MODE, LL>(s_a, bx);
        else
            forward_tile_body<32, MODE, LL>(s_a, bx);
    }
}

int resident_blocks(const void *kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

// Nonzeros of the rays of a view range: band pieces of positive length that
// fall inside the image (one thread per ray, same geometry as the projector).
__global__ void __launch_bounds__(kBlock) count_nnz_kernel(const FwdArgs a, unsigned long long *count) {
    const long long n_rays = (long long)(a.v_end - a.v_begin) * a.nb;
    const long long ray = (long long)blockIdx.x * kBlock + threadIdx.x;
    unsigned long long c = 0;
    if (ray < n_rays) {
        const int p = a.v_begin + (int)(ray / a.nb);
        const int j = (int)(ray % a.nb);
        const int v = a.order[p];
        const ViewParams vp = a.views[v];
        const float2 u = a.uc[(long long)v * a.nb + j];
        const int n_major = vp.col ? a.nx : a.ny;
        const int n_minor = vp.col ? a.ny : a.nx;
        const int ui = (int)u.x + (n_minor >> 1);
        const float hm = 0.5f * (float)n_major;
        float kc = -hm;
        float va = band_point(vp, u.y, kc);
        for (int k = 0; k < n_major; ++k) {
            kc += 1.0f;
            const float vb = band_point(vp, u.y, kc);
            float fl, w0, w1;
            band_split(vp, va, vb, fl, w0, w1);
            const int m0 = (int)fl + ui;
            c += (w0 > 0.0f && (unsigned)m0 < (unsigned)n_minor) ? 1 : 0;
            c += (w1 > 0.0f && (unsigned)(m0 + 1) < (unsigned)n_minor) ? 1 : 0;
            va = vb;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

template <int CHUNKS>
pet_status dispatch_tile(const FwdArgs &a, int mode, bool ll, int blocks, cudaStream_t s) {
    void (*k)(FwdArgs) = nullptr;
    if (mode == FWD_YHAT && !ll)
        k = forward_tile_kernel<CHUNKS, FWD_YHAT, false>;
    else if (mode == FWD_RATIO && !ll)
        k = forward_tile_kernel<CHUNKS, FWD_RATIO, false>;
    else if (mode == FWD_RATIO && ll)
        k = forward_tile_kernel<CHUNKS, FWD_RATIO, true>;
    else if (mode == FWD_NONE && ll)
        k = forward_tile_kernel<CHUNKS, FWD_NONE, true>;
    else
        return set_error(PET_ERR_INVALID, "forward: unsupported mode");
    launch_dependent(k, dim3((unsigned)blocks), dim3(kBlock), 0, s, a);
    return check_launch("forward_tile_kernel");
}

}  // namespace

pet_status launch_count_nnz(const FwdArgs &a, unsigned long long *d_count, cudaStream_t s) {
    const int n_rays = (a.v_end - a.v_begin) * a.nb;
    if (n_rays == 0) return PET_OK;
    if (a.lz) return launch_count_nnz_ring(a, d_count, s);
    count_nnz_kernel<<<(n_rays + kBlock - 1) / kBlock, kBlock, 0, s>>>(a, d_count);
    return check_launch("count_nnz_kernel");
}

int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        return v;
    }();
    return n;
}

pet_status launch_persistent_forward(const BatchMember *d_members, const WorkSeg *d_segs, int n_segs, int n_items,
                                     int iter, int in_is_img, int *claim, bool objective, cudaStream_t s) {
    if (n_items <= 0) return PET_OK;
    void (*k)(const BatchMember *, const WorkSeg *, int, int, int, int, int *) =
        objective ? persistent_forward_kernel<FWD_NONE, true> : persistent_forward_kernel<FWD_RATIO, false>;
    static const int resident[2] = {
        resident_blocks((const void *)persistent_forward_kernel<FWD_RATIO, false>, kBlock, 0),
        resident_blocks((const void *)persistent_forward_kernel<FWD_NONE, true>, kBlock, 0)};
    const int grid = std::min(n_items, resident[objective ? 1 : 0] * sm_count());
    ProfileScope prof(objective ? 3 : 0, s);
    launch_dependent(k, dim3((unsigned)grid), dim3(kBlock), 0, s, d_members, d_segs, n_segs, n_items, iter,
                     in_is_img, claim);
    return check_launch("persistent_forward_kernel");
}

__global__ void zero_ints_kernel(int *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

pet_status launch_zero_ints(int *p, int n, cudaStream_t s) {
    if (n <= 0) return PET_OK;
    zero_ints_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, n);
    return check_launch("zero_ints_kernel");
}

// Below this many blocks a multi-ring forward launch is too small to fill a
// 152-SM GB300 twice over with one block per SM.
constexpr int kSmallGrid = 2 * 152;

pet_status launch_forward(const FwdArgs &a, int mode, bool ll, int group, cudaStream_t s, int *n_blocks_out,
                          int rays_for_grid) {
    const int n_rays = rays_for_grid >= 0 ? rays_for_grid : (a.v_end - a.v_begin) * a.nb;
    // multi-ring threads carry all ring pairs of their ray; a small multi-ring
    // grid (a subset update) widens its band chunks up to 32 per ray to cut
    // each thread's chain, while full passes keep the plan's chunk count
    if (a.lz)
        while (group < 32 && forward_blocks(n_rays, 1, group) < kSmallGrid) group *= 2;
    const int blocks = a.lz ? forward_blocks(n_rays, 1, group) : forward_blocks(n_rays, a.nz, group);
    if (n_blocks_out) *n_blocks_out = blocks;
    if (blocks == 0) return PET_OK;
    ProfileScope prof(a.t_dev ? 0 : 3, s);     // 0: subset update forward, 3: full-data / API forward
    if (a.lz || a.nz > 1) return launch_forward_volume(a, mode, ll, group, blocks, s);
    if (a.nz == 1) {
        switch (group) {
            case 8: return dispatch_tile<8>(a, mode, ll, blocks, s);
            case 16: return dispatch_tile<16>(a, mode, ll, blocks, s);
            case 32: return dispatch_tile<32>(a, mode, ll, blocks, s);
            default: return set_error(PET_ERR_INVALID, "forward: unsupported lane group");
        }
    }
    return set_error(PET_ERR_INVALID, "forward: unsupported lane group");
}

}  // namespace petvr
