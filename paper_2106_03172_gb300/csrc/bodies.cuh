// The single-slice projector bodies shared by the single-state kernels, the
// persistent batched phases and the dependency-driven batched epoch: the
// forward band-chunk body (forward_tile_body) and the tiled back projection
// with its update epilogue (back_tile_body).
//
// COH: the images and ratios the body reads may have been written earlier in
// the same kernel launch (the dependency-driven epoch), so they are read with
// plain loads instead of the read-only data path.  WIDE (forward): the block
// is wider than kBlock threads; the threads past kBlock take part in the
// barriers only.
#pragma once

#include "epilogue.cuh"

namespace petvr {

namespace {

constexpr int kTile = 16;           // single slice: a block owns a kTile x kTile tile (kTile^2 == kBlock)
constexpr int kChunk = 16;          // views per shared-memory pass
constexpr int kTileBlockMax = 1024; // threads of a tile block: kTile * kTile / run per view of a chunk
// Threads of a persistent back block: one 256-thread block per tile, whose
// threads loop over the runs of subsets with more than 8 views (run 8) or 4
// views (run 4).  Measured on the 64-reconstruction batch (most members need
// 512 threads for one run per thread): 118k pairs/s at 256 threads (five
// blocks per SM), 111k at 288-320, 102k at 512 (two blocks per SM).
constexpr int kPersistentBackMax = 256;
constexpr int kPersistentBackRegs = 48;  // five 256-thread blocks per SM

// Single-slice forward: a block takes RAYS adjacent rays of the view range
// and splits each ray's bands into CHUNKS contiguous chunks (RAYS * CHUNKS =
// kBlock).  Inside a warp, lane = 8 * chunk + ray: the 32 lanes are 8
// adjacent rays times 4 chunks, so one warp load touches 4 image rows with
// 8 neighbouring pixels each.  Chunk sums are reduced by xor-shuffles
// (within the warp) and then over warps through shared memory, always in the
// same order, so the result is deterministic.
template <int CHUNKS, int MODE, bool LL, bool INTERIOR = true, bool COH = false, bool WIDE = false>
__device__ __forceinline__ void forward_tile_body(const FwdArgs &a, const int bx) {
    constexpr int RAYS = kBlock / CHUNKS;        // rays per block
    constexpr int WPG = CHUNKS / 4;              // warps per group of 8 rays
    const RayRange rr = ray_range(a);
    const int n_rays = (rr.v_end - rr.v_begin) * a.nb;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int r8 = lane & 7;
    const int chunk = 4 * (warp % WPG) + (lane >> 3);
    const int ray_local = 8 * (warp / WPG) + r8;
    const int ray = bx * RAYS + ray_local;     // 32-bit: a plan has fewer than 2^31 rays

    // the ray's geometry: plan constants only, so it may overlap the end of
    // the kernel before this one
    float acc = 0.0f;
    ViewParams vp{};
    float2 u = make_float2(0.0f, 0.0f);
    int kb = 0, ke = 0, n_minor = 0, ui = 0;
    float hm = 0.0f;
    // WIDE: a block wider than kBlock; its threads past kBlock take no ray
    if (ray < n_rays && (!WIDE || threadIdx.x < kBlock)) {
        const int q = ray / a.nb;
        const int j = ray - q * a.nb;
        const int v = __ldg(a.order + rr.v_begin + q);
        vp = a.views[v];
        u = __ldg(a.uc + (long long)v * a.nb + j);
        const int n_major = vp.col ? a.nx : a.ny;
        n_minor = vp.col ? a.ny : a.nx;
        hm = 0.5f * (float)n_major;
        ui = (int)u.x + (n_minor >> 1);
        int k_lo, k_hi;
        band_range(vp, u.x + u.y, n_major, n_minor, k_lo, k_hi);
        // chunks are aligned to the same bands for every ray of the view, so
        // neighbouring lanes read the same image rows
        const int per = (n_major + CHUNKS - 1) / CHUNKS;
        kb = max(k_lo, chunk * per);
        ke = min(k_hi, (chunk + 1) * per);
    }
    pdl_wait();
    pdl_trigger();
    // counts and background of the ray this thread finishes below: issued now
    // (they may come from the kernel before, hence after the wait) so that
    // their latency hides behind the band walk
    const int ray_f = bx * RAYS + (int)threadIdx.x;
    const bool fin = threadIdx.x < RAYS && ray_f < n_rays;
    const long long gi = rr.off + ray_f;
    float g_f = 0.0f, w_f = a.w_scalar;
    if (fin) {
        if (MODE == FWD_RATIO || LL) g_f = __ldg(a.g + gi);
        if (a.w) w_f = __ldg(a.w + gi);
    }
    {
        if (kb < ke) {
            const int s_major = vp.col ? 1 : a.nx;
            const int s_minor = vp.col ? a.nx : 1;
            float kc = (float)kb - hm;
            float va = band_point(vp, u.y, kc);
            // kBatch bands at a time: all their pixel offsets and weights
            // first, then the loads, then the FMAs in band order, so that the
            // loads of a batch are in flight together.  A piece outside the
            // image (or of a band past ke) is not loaded and adds 0 * 0,
            // which leaves acc unchanged: the sum is the same as with the
            // piece skipped.
            constexpr int kBatch = 4;
            for (int k = kb; k < ke; k += kBatch) {
                int o0[kBatch], o1[kBatch];
                float c0[kBatch], c1[kBatch];
                // Interior batch: the ray's minor position is linear in kc, so
                // every band's pieces lie between the pixels of the batch's two
                // end points, up to rounding that moves a floor by at most one.
                // With one pixel of margin on each side both pieces of every
                // band are inside the image, and the offsets need no checks
                // (they equal the checked ones).
                bool interior = false;
                if (INTERIOR) {
                    const float vend = band_point(vp, u.y, kc + (float)kBatch);
                    const int e_lo = (int)floorf(fminf(va, vend)) + ui;
                    const int e_hi = (int)floorf(fmaxf(va, vend)) + ui;
                    interior = k + kBatch <= ke && e_lo >= 1 && e_hi <= n_minor - 3;
                }
                if (interior) {
#pragma unroll
                    for (int b = 0; b < kBatch; ++b) {
                        kc += 1.0f;
                        const float vb = band_point(vp, u.y, kc);
                        float fl, w0, w1;
                        band_split(vp, va, vb, fl, w0, w1);
                        o0[b] = (k + b) * s_major + ((int)fl + ui) * s_minor;
                        o1[b] = o0[b] + s_minor;
                        c0[b] = w0;
                        c1[b] = w1;
                        va = vb;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < kBatch; ++b) {
                        kc += 1.0f;
                        const float vb = band_point(vp, u.y, kc);
                        float fl, w0, w1;
                        band_split(vp, va, vb, fl, w0, w1);
                        const int m0 = (int)fl + ui;
                        const bool live = k + b < ke;
                        const bool ok0 = live && (unsigned)m0 < (unsigned)n_minor;
                        const bool ok1 = live && w1 > 0.0f && (unsigned)(m0 + 1) < (unsigned)n_minor;
                        const int row = (k + b) * s_major;
                        o0[b] = ok0 ? row + m0 * s_minor : 0;
                        o1[b] = ok1 ? row + (m0 + 1) * s_minor : 0;
                        c0[b] = ok0 ? w0 : 0.0f;
                        c1[b] = ok1 ? w1 : 0.0f;
                        va = vb;
                    }
                }
                float x0[kBatch], x1[kBatch];
#pragma unroll
                for (int b = 0; b < kBatch; ++b) {
                    x0[b] = c0[b] != 0.0f ? ld_data<COH>(a.img + o0[b]) : 0.0f;
                    x1[b] = c1[b] != 0.0f ? ld_data<COH>(a.img + o1[b]) : 0.0f;
                }
#pragma unroll
                for (int b = 0; b < kBatch; ++b) {
                    acc = fmaf(c0[b], x0[b], acc);
                    acc = fmaf(c1[b], x1[b], acc);
                }
            }
        }
    }
    // the 4 chunks of each ray in this warp, then the warps of its group
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    __shared__ float red[kBlock / 32][8];
    if (lane < 8 && (!WIDE || warp < kBlock / 32)) red[warp][lane] = acc;
    __syncthreads();

    double ll = 0.0;
    if (threadIdx.x < RAYS) {
        const int g = threadIdx.x >> 3;
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < WPG; ++w) sum += red[g * WPG + w][threadIdx.x & 7];
        if (fin) {
            const float yhat = sum + w_f;
            if (MODE == FWD_YHAT) a.out[ray_f] = yhat;
            if (MODE == FWD_RATIO || LL) {
                const float g = g_f;
                if (MODE == FWD_RATIO) a.out[ray_f] = (yhat != 0.0f) ? g / yhat : 0.0f;
                if (LL) {
                    if (yhat > 0.0f) {
                        ll = (g > 0.0f ? (double)g * (double)logf(yhat) : 0.0) - (double)yhat;
                    } else if (g > 0.0f) {
                        // g log(yhat) with yhat <= 0 and g > 0: the objective is -inf there
                        // (latched as well when the caller gave a status word)
                        ll = -(double)INFINITY;
                        if (a.status) atomicExch(a.status, (int)PET_ERR_NUMERIC);
                    } else {
                        ll = -(double)yhat;
                    }
                }
            }
        }
    }
    if (LL) {
        __shared__ double dred[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
        if (lane == 0 && (!WIDE || warp < kBlock / 32)) dred[warp] = ll;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < kBlock / 32; ++i) s += dred[i];
            a.ll_partials[bx] = s;
        }
    }
}

// Single-slice path: a block owns a kTile x kTile pixel tile.  For each view,
// the tile's bands are cut into runs of kRun pixels along the view's minor
// axis; one thread walks the rays that can cross a run in band order and
// adds each ray's two band pieces into per-view partial sums in shared
// memory (every (view, pixel) slot has exactly one writer, so no atomics).
// Then each thread sums its pixel's partials over the views in a fixed order
// and applies the update.  Each ray-band split is evaluated once per run
// instead of once per pixel it touches.  Views are processed in chunks of
// kChunk to bound shared memory.
template <int EPI, typename TQ, int kRun, bool GENPOT, bool COH = false>
__device__ __forceinline__ void back_tile_body(const BackArgs &a, const int t, const int bx) {
    extern __shared__ unsigned char smem_raw[];
    const int vb = __ldg(a.sub_off + t);
    const int nv = __ldg(a.sub_off + t + 1) - vb;
    float *s_part = reinterpret_cast<float *>(smem_raw);                       // [kChunk][kTile*kTile]
    ViewParams *s_views = reinterpret_cast<ViewParams *>(s_part + kChunk * kTile * kTile);   // [kChunk]
    int *s_vid = reinterpret_cast<int *>(s_views + kChunk);
    const int r_view0 = a.t_dev ? vb : a.r_view0;
    const int nthr = blockDim.x;                  // >= kTile * kTile; one run per thread when nv <= nthr / 32

    const int tiles_x = (a.nx + kTile - 1) / kTile;
    const int x0 = (bx % tiles_x) * kTile;
    const int y0 = (bx / tiles_x) * kTile;
    constexpr int kRunsPerBand = kTile / kRun;
    constexpr int kRunsPerView = kTile * kRunsPerBand;

    float acc = 0.0f;
    for (int q0 = 0; q0 < nv; q0 += kChunk) {
        const int nq = min(kChunk, nv - q0);
        for (int q = threadIdx.x; q < nq; q += nthr) {
            const int v = __ldg(a.order + vb + q0 + q);
            s_vid[q] = v;
            s_views[q] = a.views[v];
        }
        for (int e = threadIdx.x; e < nq * kTile * kTile; e += nthr) s_part[e] = 0.0f;
        __syncthreads();
        if (q0 == 0) {
            // the staging above read plan constants only; the ratios and the
            // images below come from earlier kernels
            pdl_wait();
            pdl_trigger();
        }
        for (int run = threadIdx.x; run < nq * kRunsPerView; run += nthr) {
            const int ql = run / kRunsPerView;
            const int rem = run - ql * kRunsPerView;
            const int band = rem / kRunsPerBand;          // band offset inside the tile
            const int seg = rem - band * kRunsPerBand;
            const ViewParams vp = s_views[ql];
            const int v = s_vid[ql];
            const int k = (vp.col ? x0 : y0) + band;      // major index
            const int mstart = (vp.col ? y0 : x0) + seg * kRun;
            const int n_major = vp.col ? a.nx : a.ny;
            const int n_minor = vp.col ? a.ny : a.nx;
            const int mlen = min(kRun, n_minor - mstart);
            if (k >= n_major || mlen <= 0) continue;
            const int m0rel = mstart - (n_minor >> 1);
            const float kc = (float)k - 0.5f * (float)n_major;
            int jlo, jhi;
            candidate_bins(vp, kc, (float)m0rel, (float)(m0rel + mlen), a.nb, jlo, jhi);
            // local pixel index of minor offset c inside the run: row-driven runs
            // go along x, column-driven runs along y
            const int lbase = vp.col ? (seg * kRun) * kTile + band : band * kTile + seg * kRun;
            const int lstep = vp.col ? kTile : 1;
            float *pp = s_part + ql * kTile * kTile + lbase;
            const float2 *ucv = a.uc + v * a.nb;
            const float *rv = a.r + (vb + q0 + ql - r_view0) * a.nb;
            for (int j = jlo; j <= jhi; ++j) {
                const float2 u = __ldg(ucv + j);
                float fl, w0, w1;
                band_split(vp, band_point(vp, u.y, kc), band_point(vp, u.y, kc + 1.0f), fl, w0, w1);
                const int c = (int)fl + (int)u.x - m0rel;
                const float r = ld_data<COH>(rv + j);
                if ((unsigned)c < (unsigned)mlen) pp[c * lstep] += w0 * r;
                if (w1 > 0.0f && (unsigned)(c + 1) < (unsigned)mlen) pp[(c + 1) * lstep] += w1 * r;
            }
        }
        __syncthreads();
        if (threadIdx.x < kTile * kTile)
            for (int ql = 0; ql < nq; ++ql) acc += s_part[ql * kTile * kTile + threadIdx.x];
        __syncthreads();
    }
    pdl_wait();   // returns at once after the wait above; covers an empty subset
    if (threadIdx.x < kTile * kTile) {
        const int ix = x0 + (threadIdx.x % kTile);
        const int iy = y0 + (threadIdx.x / kTile);
        if (ix < a.nx && iy < a.ny) {
            const int n = iy * a.nx + ix;
            apply_epilogue<EPI, TQ, GENPOT, COH>(a, t, n, n, ix, iy, 0, acc);
        }
    }
}

}  // namespace

}  // namespace petvr
