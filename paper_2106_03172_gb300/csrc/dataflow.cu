// Dependency-driven batched epoch: one resident grid runs every update of an
// epoch call for every member of a batch.
//
// The host lists every stage of every member in order (per update: at an
// anchor update the anchor forward over all views, the anchor back projection
// over all subsets and the anchor finish, then the subset forward and the
// subset back projection + update), merges the members' lists stage by stage,
// and records for each segment the earlier segments of the same member it
// needs: a subset or anchor forward needs the previous update's back
// projection (the iterate it reads), an anchor back projection its anchor
// forward (the ratios), an anchor finish its back projection (B), and an
// update's back projection its forward (the ratios) and, at an anchor update,
// the finish (s_anc, f_anc or q~).  Blocks claim items in list order; before
// an item, thread 0 waits until each needed segment has counted all its items
// done.  Every needed segment lies earlier in the list and was claimed by a
// running block (claims are dynamic from the first item on), so the earliest
// unfinished item never waits: the waits end.
// Each wait is nevertheless bounded (a poll count set by the host); when it
// runs out the kernel latches PET_ERR_TIMEOUT in the batch's status word,
// later items skip their work, and the launch ends.
//
// Memory order: a block's item writes, a barrier, then thread 0's fence and
// atomic count (release); a waiting thread 0 reads the count with an acquire
// load, then a barrier, then the block reads.  Data written earlier in the
// launch (iterates, ratios, anchor caches) are read with plain loads (the
// bodies' COH variant), not through the read-only data path.
//
// An item is one block of the member's own single-state launch, run by the
// same body with the same launch shape, so each member's results are
// bit-identical to its own epoch calls (the finish items repeat the finish
// kernels' arithmetic).
#include <algorithm>

#include "bodies.cuh"

namespace petvr {

namespace {

constexpr int kDataflowRegs = 48;

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int find_df_segment(const DfSeg *segs, int n_segs, int g) {
    int lo = 0, hi = n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&segs[mid].first) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Thread 0: wait until done[dep] >= need.  False when another block latched an
// error, or when `limit` polls have passed (then PET_ERR_TIMEOUT is latched).
__device__ __forceinline__ bool wait_done(const int *done, int dep, int need, int *status, long long limit) {
    if (dep < 0) return true;
    for (long long it = 0; ld_acquire(done + dep) < need; ++it) {
        if (*(volatile int *)status != 0) return false;
        if (it >= limit) {
            atomicCAS(status, 0, (int)PET_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

// The anchor finishes of one pixel (the arithmetic of the finish kernels).
struct FinArgs {
    const float *B;     // [ns][plane] anchor cache
    const float *f;     // the anchor iterate
    float *f_anc, *s_anc, *s_hat, *qtil;
    const float *sens;
    int ns, nz, svrem, init;
    long long plane;
};

__device__ __forceinline__ void finish_pixel(const FinArgs &a, long long i) {
    double s = 0.0;
    for (int t = 0; t < a.ns; ++t) s += a.B[(long long)t * a.plane + i];
    if (a.svrem) {
        const float fa = a.f[i];
        a.f_anc[i] = fa;
        const float sa = (float)((double)fa * s);
        a.s_anc[i] = sa;
        if (a.init) a.s_hat[i] = sa;
    } else {
        a.qtil[i] = (float)((s - (double)a.sens[i / a.nz]) / (double)a.ns);
    }
}

template <int kRun, bool GENPOT>
__device__ __forceinline__ void df_update_tile(int algo, int table_dtype, const BackArgs &b, int t, int tile) {
    switch (algo) {
        case PET_ALGO_OSEM: back_tile_body<EPI_OSEM, float, kRun, GENPOT, true>(b, t, tile); break;
        case PET_ALGO_SVREM: back_tile_body<EPI_SVREM, float, kRun, GENPOT, true>(b, t, tile); break;
        case PET_ALGO_SAGA:
            if (table_dtype == PET_TABLE_BF16)
                back_tile_body<EPI_SAGA, __nv_bfloat16, kRun, GENPOT, true>(b, t, tile);
            else
                back_tile_body<EPI_SAGA, float, kRun, GENPOT, true>(b, t, tile);
            break;
        case PET_ALGO_SGA: back_tile_body<EPI_SGA, float, kRun, GENPOT, true>(b, t, tile); break;
        case PET_ALGO_SEM: back_tile_body<EPI_SEM, float, kRun, GENPOT, true>(b, t, tile); break;
        case PET_ALGO_SAGAEM: back_tile_body<EPI_SAGAEM, float, kRun, GENPOT, true>(b, t, tile); break;
        default: back_tile_body<EPI_SVRG, float, kRun, GENPOT, true>(b, t, tile); break;
    }
}

template <bool GENPOT>
__global__ void __maxnreg__(kDataflowRegs)
    dataflow_epoch_kernel(const BatchMember *ms, const DfSeg *segs, int n_segs, int n_items, int odd, int *done,
                          int *status, long long wait_limit) {
    __shared__ union {
        FwdArgs f;
        BackArgs b;
        FinArgs fin;
    } s_args;
    __shared__ int s_item, s_seg, s_ok, s_kind, s_shape, s_bx, s_t, s_algo, s_tq;
    int *claim = done;             // done[0]: the claim counter; done[1 + k]: items of segment k done
    int *seg_done = done + 1;
    // the counters were zeroed by the kernel ahead of this one
    pdl_wait();
    pdl_trigger();
    // every item is claimed by a running block (no block's first item is fixed
    // in advance: a block that is not yet resident holds no item anyone waits for)
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int g = atomicAdd(claim, 1);
            s_item = g;
            if (g < n_items) {
                const int k = find_df_segment(segs, n_segs, g);
                const DfSeg sg = segs[k];
                s_seg = k;
                const bool ok = *(volatile int *)status == 0 &&
                                wait_done(seg_done, sg.dep0, sg.need0, status, wait_limit) &&
                                wait_done(seg_done, sg.dep1, sg.need1, status, wait_limit);
                s_ok = ok ? 1 : 0;
                if (ok) {
                    const BatchMember &m = ms[sg.member];
                    const bool in_is_img = ((sg.iter % 2) == 0) != (odd != 0);
                    float *in = in_is_img ? m.img : m.alt;
                    float *out = in_is_img ? m.alt : m.img;
                    const int local = g - sg.first;
                    s_kind = sg.kind;
                    s_shape = sg.shape;
                    s_bx = local;
                    s_algo = m.algo;
                    s_tq = m.table_dtype;
                    if (sg.kind == DF_FWD_UPDATE || sg.kind == DF_FWD_ANCHOR) {
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
                        a.img = in;
                        if (sg.kind == DF_FWD_UPDATE) {
                            a.sub_off = m.sub_off;
                            a.t_dev = m.seq + sg.iter;
                            a.out = m.ratio;
                        } else {
                            a.v_begin = 0;
                            a.v_end = m.na;
                            a.out = m.ratio_full;
                        }
                        s_args.f = a;
                    } else if (sg.kind == DF_FINISH) {
                        FinArgs a{};
                        a.B = m.B;
                        a.f = in;
                        a.f_anc = const_cast<float *>(m.f_anc);
                        a.s_anc = const_cast<float *>(m.s_anc);
                        a.s_hat = m.s_hat;
                        a.qtil = const_cast<float *>(m.qtil);
                        a.sens = m.sens;
                        a.ns = m.ns;
                        a.nz = 1;
                        a.svrem = m.algo == PET_ALGO_SVREM;
                        a.init = sg.flag;
                        a.plane = (long long)m.nx * m.ny;
                        s_args.fin = a;
                    } else {
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
                        if (sg.kind == DF_BACK_ANCHOR) {
                            const int t = local / sg.tiles;
                            b.r = m.ratio_full;
                            b.r_view0 = 0;
                            b.out = const_cast<float *>(m.B);
                            s_t = t;
                            s_bx = local - t * sg.tiles;
                        } else {
                            b.t_dev = m.seq + sg.iter;
                            b.r = m.ratio;
                            b.f = in;
                            b.f_out = out;
                            b.sens_t = m.sens_t;
                            b.sens = m.sens;
                            b.beta = m.beta;
                            b.pot = m.pot;
                            b.delta = m.delta;
                            b.alpha = m.alpha;
                            b.alpha_dev = m.alphas ? m.alphas + sg.iter : nullptr;
                            b.s_hat = m.s_hat;
                            b.f_anc = m.f_anc;
                            b.s_anc = m.s_anc;
                            b.B = m.B;
                            b.d = m.d;
                            b.table = m.table;
                            b.qbar = m.qbar;
                            b.qtil = m.qtil;
                            s_t = __ldg(m.seq + sg.iter);
                        }
                        s_args.b = b;
                    }
                }
            }
        }
        __syncthreads();
        if (s_item >= n_items) break;
        if (s_ok) {
            const int kind = s_kind, shape = s_shape, bx = s_bx;
            if (kind == DF_FWD_UPDATE || kind == DF_FWD_ANCHOR) {
                if (shape == 8)
                    forward_tile_body<8, FWD_RATIO, false, true, true, true>(s_args.f, bx);
                else if (shape == 16)
                    forward_tile_body<16, FWD_RATIO, false, true, true, true>(s_args.f, bx);
                else
                    forward_tile_body<32, FWD_RATIO, false, true, true, true>(s_args.f, bx);
            } else if (kind == DF_FINISH) {
                const long long i = (long long)bx * kBlock + threadIdx.x;
                if (threadIdx.x < kBlock && i < s_args.fin.plane) finish_pixel(s_args.fin, i);
            } else if (kind == DF_BACK_ANCHOR) {
                if (shape == 4)
                    back_tile_body<EPI_ANCHOR, float, 4, false, true>(s_args.b, s_t, bx);
                else
                    back_tile_body<EPI_ANCHOR, float, 8, false, true>(s_args.b, s_t, bx);
            } else if (shape == 4) {
                df_update_tile<4, GENPOT>(s_algo, s_tq, s_args.b, s_t, bx);
            } else {
                df_update_tile<8, GENPOT>(s_algo, s_tq, s_args.b, s_t, bx);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(seg_done + s_seg, 1);
        }
    }
}

size_t df_smem_bytes() { return (size_t)kChunk * (kTile * kTile * sizeof(float) + sizeof(ViewParams) + sizeof(int)); }

}  // namespace

pet_status launch_dataflow_epoch(const BatchMember *d_members, const DfSeg *d_segs, int n_segs, int n_items,
                                 int odd, int *d_done, int *d_status, long long wait_limit, bool general_potential,
                                 int threads, cudaStream_t s) {
    if (n_items <= 0) return PET_OK;
    if (threads < kTile * kTile || threads > kPersistentBackMax)
        return set_error(PET_ERR_INVALID, "dataflow: block size");
    void (*k)(const BatchMember *, const DfSeg *, int, int, int, int *, int *, long long) =
        general_potential ? dataflow_epoch_kernel<true> : dataflow_epoch_kernel<false>;
    const size_t smem = df_smem_bytes();
    static int resident[2][kPersistentBackMax + 1] = {};   // blocks per SM by potential class and block size
    int &per_sm = resident[general_potential ? 1 : 0][threads];
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k, threads, smem) != cudaSuccess ||
         per_sm < 1))
        per_sm = 1;
    const int grid = std::min(n_items, per_sm * sm_count());
    launch_dependent(k, dim3((unsigned)grid), dim3((unsigned)threads), smem, s, d_members, d_segs, n_segs, n_items,
                     odd, d_done, d_status, wait_limit);
    return check_launch("dataflow_epoch_kernel");
}

}  // namespace petvr
