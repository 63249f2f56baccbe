// Back projection as a pixel-driven gather (K2), fused with the per-pixel
// update of each method (K3).
//
// b_n = sum_{m in S_t} a_mn r_m as a gather per pixel (no atomics, so the
// result is deterministic).  Single slices use tiles with runs of pixels
// that share each ray's band split (back_tile_kernel, here); slice stacks
// and multi-ring volumes have their own kernels in volume_back.cu (z-lanes
// over a pixel's slices; each band piece split over the layers its axial
// range crosses).  In each view only the bins whose ray
// can cross the pixel's major band at the pixel are candidates (usually
// 2-3), found from the bin spacing K, and each candidate's weight comes from
// band_point() / band_split(), the functions the forward kernels use, so A^T
// here is the exact transpose of A there.
//
// The epilogue then applies the method's update with b_n still in a
// register (the penalty's neighbours, 4 in a plane and 2 more along z in a
// volume, are read from f^k, §3):
//   OSEM   f' = root(a = f b, S = sens_t, beta / N_s)                (§2.2, §3)
//   SVREM  s' = (1-alpha) s + alpha (N_s f b - N_s f_anc B_t + s_anc),
//          f' = root(a = s', S = sens, beta)                        (§2.3, §3)
//   SAGA   q = b - sens_t - (beta/N_s) grad R(f);
//          f' = max(0, f + alpha d (q - q_t + qbar)); qbar += (q - q_t)/N_s;
//          q_t = q                                                  (§4)
//   SVRG   f' = max(0, f + alpha d (b - B_t - (beta/N_s) grad R(f) + q~))
//          (the anchor's penalty terms cancel against those inside q~) (§4)
//   ANCHOR B_t = b for every subset t at once (grid.y = t)
//   SAGA_INIT table_t = b - sens_t - (beta/N_s) grad R(f) for every t.
#include <algorithm>

#include "bodies.cuh"

namespace petvr {

namespace {

// The all-subset launches (anchor passes, table fills), the full-data
// statistic and plain back projections run in back_tile_wide_kernel, capped at
// 48 registers: four 288-thread blocks per SM where the compiler's own choice
// (57) leaves three.  The subset updates keep theirs (42).
constexpr bool wide_epilogue(int epi) {
    return epi == EPI_ANCHOR || epi == EPI_SAGA_INIT || epi == EPI_SAGAEM_INIT || epi == EPI_SEM_INIT ||
           epi == EPI_PLAIN;
}
constexpr int kWideRegs = 48;
static_assert(kTile * kTile == kBlock, "one pixel of the tile per thread");

template <int EPI, typename TQ, int kRun, bool GENPOT>
__global__ void __launch_bounds__(kTileBlockMax) back_tile_kernel(const BackArgs a) {
    const int t = a.t_dev ? __ldg(a.t_dev) : a.t0 + (int)blockIdx.y;
    back_tile_body<EPI, TQ, kRun, GENPOT>(a, t, blockIdx.x);
}

template <int EPI, typename TQ, int kRun, bool GENPOT>
__global__ void __maxnreg__(kWideRegs) back_tile_wide_kernel(const BackArgs a) {
    const int t = a.t_dev ? __ldg(a.t_dev) : a.t0 + (int)blockIdx.y;
    back_tile_body<EPI, TQ, kRun, GENPOT>(a, t, blockIdx.x);
}

// Member update of one tile: the member's algorithm and table type select
// the epilogue (the single-state launch's template arguments).
template <int kRun, bool GENPOT>
__device__ __forceinline__ void member_update_tile(int algo, int table_dtype, const BackArgs &b, int t, int tile) {
    switch (algo) {
        case PET_ALGO_OSEM: back_tile_body<EPI_OSEM, float, kRun, GENPOT>(b, t, tile); break;
        case PET_ALGO_SVREM: back_tile_body<EPI_SVREM, float, kRun, GENPOT>(b, t, tile); break;
        case PET_ALGO_SAGA:
            if (table_dtype == PET_TABLE_BF16)
                back_tile_body<EPI_SAGA, __nv_bfloat16, kRun, GENPOT>(b, t, tile);
            else
                back_tile_body<EPI_SAGA, float, kRun, GENPOT>(b, t, tile);
            break;
        case PET_ALGO_SGA: back_tile_body<EPI_SGA, float, kRun, GENPOT>(b, t, tile); break;
        case PET_ALGO_SEM: back_tile_body<EPI_SEM, float, kRun, GENPOT>(b, t, tile); break;
        case PET_ALGO_SAGAEM: back_tile_body<EPI_SAGAEM, float, kRun, GENPOT>(b, t, tile); break;
        default: back_tile_body<EPI_SVRG, float, kRun, GENPOT>(b, t, tile); break;
    }
}

// Persistent batched back projection + update: a resident grid whose blocks
// claim work items until the list is exhausted.  An item is one tile of a
// member's update (WK_BACK_UPDATE) or one (subset, tile) of a member's anchor
// back projection (WK_BACK_ANCHOR), run by the same body with the same run
// length as the member's own launches, so results are bit-identical to them.
// Thread 0 claims the item and writes its arguments to shared memory; the
// segment table is staged in shared memory once per block.
// GENPOT: the members of this launch use an edge-preserving potential.
template <bool GENPOT>
__global__ void __maxnreg__(kPersistentBackRegs)
    persistent_back_kernel(const BatchMember *ms, const WorkSeg *segs, int n_segs, int n_items, int iter,
                           int in_is_img, int *claim) {
    __shared__ WorkSeg s_segs[kSegSmem];
    __shared__ BackArgs s_b;
    __shared__ int s_item, s_t, s_tile, s_kind, s_shape, s_algo, s_tq;
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
                BackArgs b{};
                b.views = m.views;
                b.uc = m.uc;
                b.order = m.order;
                b.sub_off = m.sub_off;
                b.nx = m.nx;
                b.ny = m.ny;
                b.nz = 1;
                b.nb = m.nb;
                b.ns = m.ns;
                b.run = sg.shape;
                const int local = g - sg.first;
                if (sg.kind == WK_BACK_ANCHOR) {
                    const int t = local / sg.tiles;
                    b.r = m.ratio_full;
                    b.r_view0 = 0;
                    b.out = const_cast<float *>(m.B);
                    s_t = t;
                    s_tile = local - t * sg.tiles;
                } else {
                    b.t_dev = m.seq + iter;
                    b.r = m.ratio;
                    b.f = in_is_img ? m.img : m.alt;
                    b.f_out = in_is_img ? m.alt : m.img;
                    b.sens_t = m.sens_t;
                    b.sens = m.sens;
                    b.beta = m.beta;
                    b.pot = m.pot;
                    b.delta = m.delta;
                    b.alpha = m.alpha;
                    b.alpha_dev = m.alphas ? m.alphas + iter : nullptr;
                    b.s_hat = m.s_hat;
                    b.f_anc = m.f_anc;
                    b.s_anc = m.s_anc;
                    b.B = m.B;
                    b.d = m.d;
                    b.table = m.table;
                    b.qbar = m.qbar;
                    b.qtil = m.qtil;
                    s_t = __ldg(m.seq + iter);
                    s_tile = local;
                }
                s_b = b;
                s_kind = sg.kind;
                s_shape = sg.shape;
                s_algo = m.algo;
                s_tq = m.table_dtype;
            }
        }
        __syncthreads();
        if (s_item >= n_items) break;
        const int t = s_t, tile = s_tile;
        if (s_kind == WK_BACK_ANCHOR) {
            if (s_shape == 4)
                back_tile_body<EPI_ANCHOR, float, 4, false>(s_b, t, tile);
            else
                back_tile_body<EPI_ANCHOR, float, 8, false>(s_b, t, tile);
        } else if (s_shape == 4) {
            member_update_tile<4, GENPOT>(s_algo, s_tq, s_b, t, tile);
        } else {
            member_update_tile<8, GENPOT>(s_algo, s_tq, s_b, t, tile);
        }
    }
}

size_t back_smem_bytes() { return (size_t)kChunk * (kTile * kTile * sizeof(float) + sizeof(ViewParams) + sizeof(int)); }

// Single-slice back-projection launch of one epilogue / table type / potential.
struct TileBack {
    const BackArgs &a;
    int ny_grid;
    cudaStream_t s;
    int max_views;

    template <int EPI, typename TQ, bool GENPOT>
    pet_status run() const {
        const int tiles = ((a.nx + kTile - 1) / kTile) * ((a.ny + kTile - 1) / kTile);
        const dim3 grid((unsigned)tiles, (unsigned)ny_grid);
        const size_t smem = back_smem_bytes();
        // one thread per run: kTile * kTile / run runs per view of the largest chunk
        const int run = a.run == 4 ? 4 : 8;
        const int per_view = kTile * (kTile / run);
        // subset launches are latency-bound: one run per thread; the all-subset and
        // full-data launches are throughput-bound: 256-thread blocks whose threads
        // loop over the runs, so that more blocks fit per SM (anchor 41.3 -> 39.5 us)
        const int threads = (wide_epilogue(EPI) && EPI != EPI_PLAIN)
                                ? kTile * kTile
                                : max(kTile * kTile, per_view * min(max_views, kChunk));
        void (*k)(BackArgs) = nullptr;
        if constexpr (wide_epilogue(EPI))
            k = run == 4 ? back_tile_wide_kernel<EPI, TQ, 4, GENPOT> : back_tile_wide_kernel<EPI, TQ, 8, GENPOT>;
        else
            k = run == 4 ? back_tile_kernel<EPI, TQ, 4, GENPOT> : back_tile_kernel<EPI, TQ, 8, GENPOT>;
        launch_dependent(k,
                         grid, dim3((unsigned)threads), smem, s, a);
        return check_launch("back_tile_kernel");
    }
};

}  // namespace

int back_block_threads(int run, int max_views) {
    const int per_view = kTile * (kTile / (run == 4 ? 4 : 8));
    return std::min(kPersistentBackMax, std::max(kTile * kTile, per_view * std::min(max_views, kChunk)));
}

pet_status launch_persistent_back(const BatchMember *d_members, const WorkSeg *d_segs, int n_segs, int n_items,
                                  int iter, int in_is_img, int *claim, bool general_potential, int threads,
                                  cudaStream_t s) {
    if (n_items <= 0) return PET_OK;
    void (*k)(const BatchMember *, const WorkSeg *, int, int, int, int, int *) =
        general_potential ? persistent_back_kernel<true> : persistent_back_kernel<false>;
    const size_t smem = back_smem_bytes();
    if (threads < kTile * kTile || threads > kPersistentBackMax)
        return set_error(PET_ERR_INVALID, "back: block size");
    static int resident[2][kPersistentBackMax + 1] = {};   // blocks per SM by potential class and block size
    int &per_sm = resident[general_potential ? 1 : 0][threads];
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k, threads, smem) != cudaSuccess ||
         per_sm < 1))
        per_sm = 1;
    const int grid = std::min(n_items, per_sm * sm_count());
    ProfileScope prof(1, s);
    launch_dependent(k, dim3((unsigned)grid), dim3((unsigned)threads), smem, s, d_members, d_segs, n_segs, n_items,
                     iter, in_is_img, claim);
    return check_launch("persistent_back_kernel");
}

pet_status launch_back(const BackArgs &a, int epi, int table_dtype, int n_subsets_grid,
                       cudaStream_t s, int max_views) {
    ProfileScope prof(n_subsets_grid > 1 ? 2 : 1, s);
    if (a.axial || a.nz > 1) return launch_back_volume(a, epi, table_dtype, n_subsets_grid, s, max_views);
    return with_epilogue(epi, table_dtype, a.pot, TileBack{a, n_subsets_grid, s, max_views});
}

}  // namespace petvr
