// Internal declarations of libpetvr: object layouts, kernel argument blocks,
// the shared ray-geometry device functions and the launch helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <utility>
#include <vector>

#include "petvr.h"

namespace petvr {

// ---------------------------------------------------------------------------
// Ray geometry.
//
// For each view the traversal runs along the "major" image axis: rows (y)
// when |cos theta| >= |sin theta|, columns (x) otherwise.  Along that axis
// the line x cos + y sin = s moves by |du| <= 1 pixel in the "minor"
// coordinate per pixel step, so inside one major step (one row band, or one
// column band) it meets at most two pixels.  The part of the line inside a
// major band has length L = d / max(|cos|, |sin|); if the band contains a
// minor grid line at position c+1 the line is split there, the first piece
// having length (c + 1 - u_lo) * Lm with Lm = L / |du|.  These are exactly
// the Siddon intersection lengths (every piece between consecutive grid-line
// crossings, charged to the pixel containing it), enumerated band by band.
//
// Minor coordinates u are in pixel units relative to the pixel edge nearest
// the image centre (u in [-mo, n_minor - mo) is inside the image, with
// mo = n_minor / 2), so that floor(u) + mo is the pixel index and axis-
// aligned rays on grid lines land on integers exactly (half-open pixels: the
// +x / +y pixel takes a ray lying on their shared edge).
//
// Precision: near-axis views (|du| small) turn an error e in u into an error
// e / |du| in where the ray crosses the nearly parallel grid line.  Each ray
// therefore carries its offset as an integer ui plus a fraction uf in
// [-1/2, 1/2] (both from FP64 on the host), the slope as du + du_lo (FP32
// value and its FP64 rounding residual), and u - ui is evaluated as
// uf + kc (du + du_lo), whose magnitude stays small exactly when |du| is.
// ---------------------------------------------------------------------------
struct ViewParams {
    float du;     // minor displacement (pixels) per major step (FP32 value)
    float du_lo;  // FP64 residual du_exact - du
    float L;      // ray length (mm) per major step
    float Lm;     // ray length (mm) per pixel of minor displacement (0 if du == 0)
    float K;      // minor displacement (pixels) per bin step (never 0)
    float invK;   // 1 / K
    float inv_du; // 1 / du (0 if du == 0), for band ranges only
    float uc0;    // centred minor coordinate of bin 0 at the central major line (approx.)
    int col;      // 1: major axis is x (columns); 0: major axis is y (rows)
};

// Bands [k_lo, k_hi) where a ray with centred minor offset uc can meet the
// image (a superset with one band of margin each side; extra bands add 0).
__device__ __forceinline__ void band_range(const ViewParams &vp, float uc, int n_major, int n_minor, int &k_lo,
                                           int &k_hi) {
    const int mo = n_minor >> 1;
    k_lo = 0;
    k_hi = n_major;
    if (vp.du == 0.0f) {
        if (!(uc >= (float)(-mo) && uc < (float)(n_minor - mo))) k_hi = 0;
        return;
    }
    const float hm = 0.5f * (float)n_major;
    const float ka = fmaf((float)(-mo - 1) - uc, vp.inv_du, hm);
    const float kb = fmaf((float)(n_minor - mo + 1) - uc, vp.inv_du, hm);
    const float kmax = (float)n_major + 1.0f;
    const float klo = fminf(fmaxf(fminf(ka, kb), -1.0f), kmax);
    const float khi = fmaxf(fminf(fmaxf(ka, kb), kmax), -1.0f);
    k_lo = max(0, (int)floorf(klo) - 1);
    k_hi = min(n_major, (int)ceilf(khi) + 1);
}

// Fractional minor position u - ui of a ray at band boundary kc (centred
// major coordinate).  Both projectors evaluate exactly this expression.
__device__ __forceinline__ float band_point(const ViewParams &vp, float uf, float kc) {
    return fmaf(kc, vp.du, fmaf(kc, vp.du_lo, uf));
}

// Split of one major band between the two minor pixels it can touch, given
// the fractional positions va, vb at its two boundaries: pixel fl (relative
// to ui) gets w0, pixel fl + 1 gets w1.  Forward and back projection both call
// this, so a_mn is bit-identical in the two directions.
__device__ __forceinline__ void band_split(const ViewParams &vp, float va, float vb, float &fl, float &w0,
                                           float &w1) {
    const float lo = fminf(va, vb);
    const float hi = fmaxf(va, vb);
    fl = floorf(lo);
    if (hi <= fl + 1.0f) {
        w0 = vp.L;
        w1 = 0.0f;
    } else {
        w0 = fminf((fl + 1.0f - lo) * vp.Lm, vp.L);
        w1 = vp.L - w0;
    }
}

// ---------------------------------------------------------------------------
// Multi-ring lines of response.  A line's transaxial part is a 2-D ray, walked
// band by band as above; along it z is linear in the centred major
// coordinate kc, and in layer units (zeta = (z - z_min) / slice) each line
// carries zeta(kc) = lz.x + lz.y * kc and the 3-D length per transaxial mm
// lz.z = sqrt(1 + kappa^2) (FP64 on the host).  Inside band [kc, kc + 1] the
// piece in minor pixel fl occupies the band fraction [f_lo, f_hi] below
// (pixel fl + 1 the rest); a piece is shared between the layers its zeta
// range crosses in proportion to the overlap.  Both projectors evaluate
// exactly these expressions, so the 3-D A^T is the exact transpose of A.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void piece_fraction(const ViewParams &vp, float w0, float w1, bool upper, float &f_lo,
                                               float &f_hi) {
    if (w1 == 0.0f) {                       // the band lies in one pixel
        f_lo = 0.0f;
        f_hi = 1.0f;
        return;
    }
    // share of pixel fl (fast division: no slow-path call; both projectors
    // evaluate this same expression, so the transpose stays exact)
    const float f0 = __fdividef(w0, vp.L);
    // du > 0: the minor coordinate grows with kc, pixel fl comes first
    const bool first = (vp.du > 0.0f) != upper;
    f_lo = first ? 0.0f : (upper ? f0 : 1.0f - f0);
    f_hi = first ? (upper ? 1.0f - f0 : f0) : 1.0f;
}

__device__ __forceinline__ float piece_zeta(const float4 &lz, float kc, float f) { return fmaf(lz.y, kc + f, lz.x); }

// Share of the axial range between za and zb (layer units) inside layer iz;
// a flat piece lies wholly in layer floor(za) (half-open layers).
__device__ __forceinline__ float layer_fraction(float za, float zb, int iz) {
    const float lo = fminf(za, zb), hi = fmaxf(za, zb);
    if (!(hi > lo)) return floorf(lo) == (float)iz ? 1.0f : 0.0f;
    const float ov = fminf(hi, (float)(iz + 1)) - fmaxf(lo, (float)iz);
    return ov > 0.0f ? __fdividef(ov, hi - lo) : 0.0f;
}

// Nonnegative root of a/f - 2 b f + c = 0 (the surrogate M-step of §3,
// Eq. (svrsurder)); cancellation-free in both signs of c, b = 0 allowed;
// 0 when S <= 0 or a <= 0 (zero-denominator remedy of §2.3).
__device__ __forceinline__ float m_step_root(float a, float S, float b, float c) {
    if (!(S > 0.0f) || !(a > 0.0f)) return 0.0f;
    const float D = sqrtf(fmaf(c, c, 8.0f * a * b));
    return (c <= 0.0f) ? (2.0f * a) / (D - c) : (c + D) / (4.0f * b);
}

// Pairwise potentials of Table 1 (t = f_n - f_j, delta > 0): rho, rho' and
// the curvature gamma = rho'(t)/t with its finite limit 1 at t = 0.  The
// hyperbola is delta^2 (sqrt(1 + (t/delta)^2) - 1), the form whose derivative
// is the printed rho' (the printed rho lacks a factor delta).
__device__ __forceinline__ void potential_dg(int pot, float delta, float t, float &drho, float &gam) {
    if (pot == PET_POT_HUBER) {
        const float a = fabsf(t);
        drho = fminf(fmaxf(t, -delta), delta);
        gam = a <= delta ? 1.0f : delta / a;
    } else if (pot == PET_POT_LOGCOSH) {
        const float th = tanhf(t / delta);
        drho = delta * th;
        gam = t != 0.0f ? delta * th / t : 1.0f;
    } else if (pot == PET_POT_HYPERBOLA) {
        const float q = t / delta;
        gam = rsqrtf(fmaf(q, q, 1.0f));
        drho = t * gam;
    } else {
        drho = t;
        gam = 1.0f;
    }
}

__device__ __forceinline__ float potential_rho(int pot, float delta, float t) {
    if (pot == PET_POT_HUBER) {
        const float a = fabsf(t);
        return a <= delta ? 0.5f * t * t : delta * a - 0.5f * delta * delta;
    }
    if (pot == PET_POT_LOGCOSH) {
        // delta^2 log cosh(t/delta) = delta^2 (|u| + log1p(exp(-2|u|)) - log 2)
        const float u = fabsf(t / delta);
        return delta * delta * (u + log1pf(expf(-2.0f * u)) - 0.69314718055994531f);
    }
    if (pot == PET_POT_HYPERBOLA) {
        const float q = t / delta;
        return delta * delta * (sqrtf(fmaf(q, q, 1.0f)) - 1.0f);
    }
    return 0.5f * t * t;
}


// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90 and later).  A projector launched
// through launch_dependent() may start while the kernel before it on the
// stream is still running: before pdl_wait() it reads only plan constants
// (views, ray offsets, subset tables, the subset sequence), and pdl_wait()
// blocks until that kernel has completed and its writes are visible.  Right
// after its own wait it calls pdl_trigger(), so the next projector's blocks
// can be scheduled and run their constant-only prologue; by then every
// kernel before this one has completed, so whatever that prologue reads was
// written before it started.  Launched the ordinary way, both are no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

bool use_pdl();   // false when PETVR_NO_PDL is set (or while per-launch profiling is on)

template <typename... Params, typename... Args>
cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = use_pdl() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Kernel argument blocks.
// ---------------------------------------------------------------------------
enum FwdMode { FWD_NONE = 0, FWD_YHAT = 1, FWD_RATIO = 2 };

struct FwdArgs {
    const ViewParams *views;  // [n_angles]
    const float2 *uc;         // [n_angles * n_bins] (ui, uf) centred minor offset per ray
    const int *order;         // view order the ray range indexes
    int v_begin, v_end;       // view positions [v_begin, v_end) of `order`
    const int *t_dev;         // if set: subset index on the device; the range is
    const int *sub_off;       //   [sub_off[t], sub_off[t+1]) and g / w are the full
                              //   subset-major arrays (offset applied on the device)
    int nx, ny, nz, nb;       // nz: entries per (view, bin): slices, or ring pairs (lz set)
    int layers;               // multi-ring: image layers (voxel index = pixel * layers + iz)
    const float4 *lz;         // multi-ring: axial table per line, [view][bin][pair]; else null
    const float *img;         // [ny][nx][nz] ([ny][nx][layers] multi-ring)
    const float *g;           // counts of these rays (compact), FWD_RATIO / LL only
    const float *w;           // background of these rays (compact) or null
    float w_scalar;
    float *out;               // compact output (yhat or ratio)
    double *ll_partials;      // per-block partial log-likelihood (LL only)
    int *status;              // device error latch (may be null)
};

// View range of a forward launch: given on the host, or (t_dev set) read on
// the device from the subset offsets, with the element offset of the range's
// first ray into the subset-major counts / background.
struct RayRange {
    int v_begin, v_end;
    long long off;   // element offset of the range's first ray in g / w (compact layouts)
};

__device__ __forceinline__ RayRange ray_range(const FwdArgs &a) {
    RayRange r;
    if (a.t_dev) {
        const int t = __ldg(a.t_dev);
        r.v_begin = __ldg(a.sub_off + t);
        r.v_end = __ldg(a.sub_off + t + 1);
        r.off = (long long)r.v_begin * a.nb * a.nz;
    } else {
        r.v_begin = a.v_begin;
        r.v_end = a.v_end;
        r.off = 0;
    }
    return r;
}

// Slice stacks (the geometry is shared by every slice): a warp of the forward
// is kStackChunks band chunks x 8 z-lanes, one of the back projection
// kStackPixels pixels x 8 z-lanes, and a z-lane carries stack_lane_slices(nz)
// slices (a window of 8 times that many per warp; deeper stacks take several
// windows).
constexpr int kStackChunks = 4;
constexpr int kStackPixels = 4;
inline int stack_lane_slices(int nz) { return nz <= 16 ? 2 : nz <= 32 ? 4 : nz <= 48 ? 6 : 8; }
inline int stack_windows(int nz) { return (nz + 8 * stack_lane_slices(nz) - 1) / (8 * stack_lane_slices(nz)); }

enum BackEpi {
    EPI_PLAIN = 0,       // out = A_t^T r
    EPI_OSEM = 1,        // penalised OSEM M-step
    EPI_SVREM = 2,       // SVREM statistic update + M-step
    EPI_SAGA = 3,        // SAGA step (table dtype is a template parameter)
    EPI_SVRG = 4,        // SVRG step
    EPI_ANCHOR = 5,      // B[t] = A_t^T r_t for every t (grid.y = subset)
    EPI_SAGA_INIT = 6,   // table[t] = grad Phi_t(f) for every t (grid.y = subset)
    EPI_SGA = 7,         // preconditioned gradient step (SGA / BSREM)
    EPI_SEM = 8,         // stochastic EM statistic update + M-step
    EPI_SEM_INIT = 9,    // s_hat = f . A^T r over all views
    EPI_SAGAEM = 10,     // SAGA on the EM statistic + M-step
    EPI_SAGAEM_INIT = 11,  // table[t] = tau_t(f) for every t (grid.y = subset)
};

struct BackArgs {
    const ViewParams *views;
    const float2 *uc;
    const int *order;
    const int *sub_off;   // view offsets of subsets in `order`
    int t0;               // subset of blockIdx.y == 0
    const int *t_dev;     // if set: the subset index is read here (grid.y must be 1)
    int run;              // single-slice tile kernel: pixels per run (4 or 8)
    int r_view0;          // view position of r[0] (ignored when t_dev is set: r is
                          //   then the compact ratio of subset *t_dev)
    int nx, ny, nz, nb, ns;  // nz: image entries per pixel (slices, or layers when axial)
    int axial;            // multi-ring: layers are coupled (6-neighbourhood penalty) and the
                          //   sensitivities are per voxel ([ns][nx*ny*nz]); else per pixel
    int pairs;            // multi-ring: sinogram entries per (view, bin)
    const float4 *lz;     // multi-ring: axial table per line, [view][bin][pair]
    const float *r;       // ratio / sinogram, [view pos - r_view0][bin][z] ([..][bin][pair])
    float *out;           // EPI_PLAIN: image; EPI_ANCHOR: B [ns][N*nz]
    // update inputs
    const float *f;       // current iterate f^k
    float *f_out;         // next iterate f^{k+1}
    const float *sens_t;  // [ns][N] subset sensitivities
    const float *sens;    // [N] full sensitivity
    float beta;           // penalty weight beta (full)
    int pot;              // potential (PET_POT_*)
    float delta;          // its transition parameter
    float alpha;
    const float *alpha_dev;  // if set: this update's step size (device), else alpha
    float *s_hat;         // SVREM / SEM running statistic
    const float *f_anc;   // SVREM anchor image
    const float *s_anc;   // SVREM anchor statistic
    const float *B;       // SVREM/SVRG cached A_t^T r_t(f_anc), [ns][N*nz]
    const float *d;       // SAGA/SVRG constant preconditioner; null: d_t(f^k) = f^k / sens_t
    void *table;          // SAGA table [ns][N*nz] (float or bf16)
    float *qbar;          // SAGA running mean of the table
    const float *qtil;    // SVRG full-gradient term
};

// One member of a batched update (device-resident descriptor): where its
// plan, problem and state live, and its subset indices for the current call.
struct BatchMember {
    const ViewParams *views;
    const float2 *uc;
    const int *order;
    const int *sub_off;
    int nx, ny, nb, ns;
    const float *sens_t;
    const float *sens;
    const float *g;
    const float *w;
    float w_scalar;
    float beta;
    int pot;
    float delta;
    int *status;
    int algo, table_dtype;
    float *img, *alt, *ratio;
    float *ratio_full;     // anchor-pass ratio over all views (SVREM, SVRG), subset-major
    float *s_hat;
    const float *f_anc, *s_anc, *B, *d;
    void *table;
    float *qbar;
    const float *qtil;
    float alpha;
    const int *seq;
    const float *alphas;   // this member's step size per update of the current call
    int na;                // views (full-data passes)
    int n_ll;              // forward blocks of a full pass (objective partial count)
    double *part;          // objective partials of this member
    double *phi;           // objective output {Phi, L, R}
};

// ---------------------------------------------------------------------------
// Persistent batched kernels: one resident grid per phase of a batched update
// (the subset forward projections, the anchor passes, the back projections +
// updates) pulls work items from a list.  The list is a sequence of segments,
// each a run of items of one member and one kind; an item is one block's
// worth of the single-state kernels (a block of rays of a forward pass, a
// 16 x 16 tile of a back projection), so every member gets bit-identical
// results to its own epoch calls.  Blocks claim items in list order with an
// atomic counter (zeroed before each phase's launch); nothing waits on
// another block, so the only ordering is the kernel boundary between phases.
// ---------------------------------------------------------------------------
enum WorkKind {
    WK_FWD_UPDATE = 0,     // rays of the member's current subset -> ratio (subset index on the device)
    WK_FWD_ANCHOR = 1,     // rays of every view -> ratio_full (anchor pass)
    WK_FWD_OBJECTIVE = 2,  // rays of every view -> log-likelihood block partials
    WK_BACK_UPDATE = 3,    // tile of the member's update (its method's epilogue)
    WK_BACK_ANCHOR = 4,    // (subset, tile) of the anchor back projection -> B
};

struct WorkSeg {
    int member;   // index into the batch's member descriptors
    int kind;     // WorkKind
    int first;    // list index of the segment's first item
    int count;    // items in the segment
    int shape;    // forward: band chunks per ray; back: pixels per run
    int tiles;    // back: tiles per subset (anchor item = t * tiles + tile)
};

// Dependency-driven batched epoch: one resident grid runs every update of an
// epoch call for all members.  Its work list holds every stage of every
// member (subset forward, subset back + update, and at anchor updates the
// anchor forward, anchor back projection and anchor finish), ordered stage by
// stage across members.  A segment's items wait (thread 0, bounded) until the
// segments it depends on - earlier stages of the same member - have counted
// all their items done; every dependency lies earlier in the list, and items
// are claimed in list order, so the earliest unfinished item never waits.
enum DfKind {
    DF_FWD_UPDATE = 0,   // ray blocks of the member's subset of update `iter` -> ratio
    DF_FWD_ANCHOR = 1,   // ray blocks of all views -> ratio_full
    DF_BACK_UPDATE = 2,  // tiles of update `iter` (the member's epilogue)
    DF_BACK_ANCHOR = 3,  // (subset, tile) items of the anchor back projection -> B
    DF_FINISH = 4,       // 256-pixel blocks of the anchor finish (SVREM s_anc / SVRG q~)
};

struct DfSeg {
    int member;   // index into the batch's member descriptors
    int kind;     // DfKind
    int first;    // list index of the segment's first item
    int count;    // items in the segment
    int shape;    // forward: band chunks per ray; back: pixels per run
    int tiles;    // back: tiles per subset
    int iter;     // the update this stage belongs to
    int flag;     // DF_FINISH of SVREM: s_hat is initialised from this anchor
    int dep0, need0;   // segment waited for (-1: none) and its item count
    int dep1, need1;
};

// Segments a persistent block stages in shared memory (longer tables are
// searched in global memory).
constexpr int kSegSmem = 160;

// Segment holding list item g (segments are sorted by `first`).
__device__ __forceinline__ int find_segment(const WorkSeg *segs, int n_segs, int g) {
    int lo = 0, hi = n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].first <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}


// ---------------------------------------------------------------------------
// Host objects.
// ---------------------------------------------------------------------------
}  // namespace petvr

struct pet_plan {
    pet_geometry geom;
    int nx, ny, nz, na, nb, ns;     // nz: independent slices (1 for a multi-ring volume)
    int N, M;                       // pixels and rays of one slice; multi-ring: voxels and lines
    int ring = 0;                   // multi-ring scanner (fully 3-D lines of response)
    int layers = 1;                 // multi-ring: image layers
    int pairs = 1;                  // multi-ring: ring pairs (lines per ray)
    int max_sub_views;
    int device;
    int fwd_chunks = 0;             // single-slice forward: band chunks per ray (8, 16 or 32)
    int back_run = 8;               // single-slice back projection: pixels per run (4 or 8)
    std::vector<int> order;         // subset-major view order
    std::vector<int> sub_off;       // [ns + 1]
    std::vector<long long> nnz;     // [ns] nonzeros of A_t (one slice)
    petvr::ViewParams *d_views = nullptr;
    float2 *d_uc = nullptr;
    int *d_order = nullptr;         // subset-major
    int *d_natural = nullptr;       // identity
    int *d_sub_off = nullptr;       // [ns + 1]
    int *d_all_off = nullptr;       // {0, na}
    float *d_sens_t = nullptr;      // [ns][N]
    float *d_sens = nullptr;        // [N]
    float4 *d_lz = nullptr;         // multi-ring: axial table per line [view][bin][pair]
};

struct pet_problem {
    const pet_plan *plan;
    pet_penalty pen;
    float w_scalar;
    float *d_g = nullptr;           // [M * nz], subset-major
    float *d_w = nullptr;           // [M * nz], subset-major, or null
    float *d_ratio = nullptr;       // [M * nz] scratch for full passes
    float *d_alt = nullptr;         // [N * nz] scratch image (warm start)
    double *d_part = nullptr;       // reduction partials
    int n_part = 0;
    double *d_scalar = nullptr;     // [4 + nz] reduction results
    int *d_status = nullptr;        // device error latch
    uint64_t version = 0;           // bumped by pet_problem_update (graphs hold w_scalar by value)
};

struct pet_batch;

struct pet_state {
    const pet_problem *prob;
    int algo, table_dtype;
    float *img;                     // caller's image (current iterate)
    float *alt = nullptr;           // ping-pong partner
    float *ratio = nullptr;         // [max subset rays * nz]
    float *ratio_full = nullptr;    // [M * nz] anchor-pass ratio (SVREM, SVRG)
    float *s_hat = nullptr, *f_anc = nullptr, *s_anc = nullptr;
    float *B = nullptr, *d = nullptr, *qbar = nullptr, *qtil = nullptr;
    void *table = nullptr;
    long long k = 0;
    int precond = PET_PRECOND_CONSTANT;   // SAGA / SVRG: d(f^(0)) or d_t(f^k)
    size_t bytes = 0;
    bool s_hat_ready = false;       // SVREM: s_hat initialised by the first anchor
    int *d_seq = nullptr;           // device copy of the current call's subset sequence
    float *d_alpha = nullptr;       // and of its step size per update
    int seq_cap = 0;
    double *d_part = nullptr;       // objective reduction scratch of this state
    int n_part = 0;
    cudaStream_t cap = nullptr;     // private stream for graph capture
    struct Graph {
        std::vector<int64_t> key;
        cudaGraphExec_t exec;
        uint64_t kernels;           // kernel nodes, counted at capture
        uint64_t last_use;          // graph_tick of its latest launch
    };
    std::vector<Graph> graphs;      // captured epochs / objectives, at most kMaxGraphs (least recently used go)
    uint64_t graph_tick = 0;
    uint64_t graph_version = 0;     // problem version the captured graphs were made with
};

struct pet_batch {
    std::vector<pet_state *> states;
    std::vector<petvr::BatchMember> members;   // host copy; uploaded before every call
    petvr::BatchMember *d_members = nullptr;
    // persistent phases of the current call: per update, the launches in order
    struct Phase {
        int kind;                   // 0 forward, 1 back + update (GENPOT 0/1 in `genpot`), 2 anchor finishes
        int seg_off, n_segs, n_items;
        int threads;                // back: block size
        int genpot;                 // back: general-potential epilogues
        int claim;                  // claim counter slot
    };
    std::vector<std::vector<Phase>> phases;   // [n_iter]
    std::vector<petvr::WorkSeg> h_segs;
    petvr::WorkSeg *d_segs = nullptr;
    int seg_cap = 0;
    int *d_claims = nullptr;        // claim counters of the current call's phases
    int claim_cap = 0;
    int n_claims = 0;
    int mode = 0;                   // 0: persistent phases, 1: dependency-driven epoch, 2: member graphs on streams
    std::vector<cudaStream_t> side; // mode 2: the batch's own streams, member j on side[j % side.size()]
    std::vector<cudaEvent_t> side_ev;
    cudaEvent_t fork_ev = nullptr;
    long long wait_limit = 1LL << 22;        // dependency-driven epoch: polls of a wait before PET_ERR_TIMEOUT
    std::vector<petvr::DfSeg> h_df;
    petvr::DfSeg *d_df = nullptr;
    int df_cap = 0;
    int *d_df_done = nullptr;       // claim counter, then one done counter per segment
    int df_done_cap = 0;
    int *d_status = nullptr;        // the batch's latched device status (PET_ERR_TIMEOUT)
    petvr::WorkSeg *d_obj_segs = nullptr;   // objective pass: every member's rays (fixed at creation)
    int n_obj_segs = 0, n_obj_items = 0;
    int *d_obj_claim = nullptr;
    bool graphs_on = true;
    int *d_seqs = nullptr;          // [n][seq_cap] subset indices of the current call
    float *d_alphas = nullptr;      // [n][seq_cap] step sizes of the current call
    int seq_cap = 0;
    cudaStream_t cap = nullptr;
    std::vector<pet_state::Graph> graphs;
    uint64_t graph_tick = 0;        // LRU clock of `graphs` (kept across the holder swaps)
};

namespace petvr {

// Launch accounting and error reporting.
extern std::atomic<uint64_t> g_launches;
// Optional event timing of kernel kinds (0 forward, 1 back+update, 2 multi-subset back).
struct ProfileScope {
    int kind;
    cudaStream_t stream;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ProfileScope(int kind, cudaStream_t s);
    ~ProfileScope();
};
pet_status set_error(pet_status code, const std::string &msg);
pet_status check_launch(const char *what);
bool profiling_enabled();

// Kernel launchers (forward.cu / backward.cu / misc.cu).
// Volumes (volume.cu): slice stacks and multi-ring scanners.
pet_status launch_forward_volume(const FwdArgs &a, int mode, bool ll, int group, int blocks, cudaStream_t s);
pet_status launch_back_volume(const BackArgs &a, int epi, int table_dtype, int n_subsets_grid, cudaStream_t s,
                              int max_views);
pet_status launch_count_nnz_ring(const FwdArgs &a, unsigned long long *d_count, cudaStream_t s);
pet_status launch_forward(const FwdArgs &a, int mode, bool ll, int group, cudaStream_t s,
                          int *n_blocks_out, int rays_for_grid = -1);
int forward_blocks(int n_rays, int nz, int group);
int choose_group(const pet_plan *plan);
int full_group(const pet_plan *plan);     // band chunks of a full-data single-slice pass
int default_chunks(int nx, int ny);
pet_status launch_back(const BackArgs &a, int epi, int table_dtype, int n_subsets_grid,
                       cudaStream_t s, int max_views);
pet_status launch_permute_sino(const float *src, float *dst, const int *order, int na, int nb, int nz,
                               cudaStream_t s);
pet_status launch_sum_sens(const float *sens_t, float *sens, int ns, int N, cudaStream_t s);
// `sums`: nz + 1 doubles of scratch (null: the problem's own, which concurrent
// warm starts of one problem must not share)
pet_status launch_uniform_image(const pet_problem *p, float *img, cudaStream_t s, double *sums = nullptr);
pet_status launch_objective_finish(const pet_problem *p, const float *img, int n_ll_blocks,
                                   double *part, double *d_out, cudaStream_t s);
pet_status launch_objective_finish_raw(int nx, int ny, int nz, float beta, const float *img, int n_ll_blocks,
                                       double *part, double *d_out, cudaStream_t s);
pet_status launch_count_nnz(const FwdArgs &a, unsigned long long *d_count, cudaStream_t s);
// Persistent phases (forward.cu / backward.cu): objective = false runs the
// ratio kinds (WK_FWD_UPDATE, WK_FWD_ANCHOR), true the log-likelihood kind.
pet_status launch_persistent_forward(const BatchMember *d_members, const WorkSeg *d_segs, int n_segs, int n_items,
                                     int iter, int in_is_img, int *claim, bool objective, cudaStream_t s);
pet_status launch_persistent_back(const BatchMember *d_members, const WorkSeg *d_segs, int n_segs, int n_items,
                                  int iter, int in_is_img, int *claim, bool general_potential, int threads,
                                  cudaStream_t s);
pet_status launch_zero_ints(int *p, int n, cudaStream_t s);
// Dependency-driven batched epoch (dataflow.cu): the whole list in one launch.
pet_status launch_dataflow_epoch(const BatchMember *d_members, const DfSeg *d_segs, int n_segs, int n_items,
                                 int odd, int *d_done, int *d_status, long long wait_limit, bool general_potential,
                                 int threads, cudaStream_t s);
int back_block_threads(int run, int max_views);   // block size a back projection of this shape needs
int sm_count();
pet_status launch_batch_objective_finish(const BatchMember *d_members, int n_members, int pen_blocks,
                                         cudaStream_t s);
pet_status launch_svrem_anchor_finish(const float *B, int ns, long long plane, int nz, const float *f,
                                      float *f_anc, float *s_anc, float *s_hat, bool init, cudaStream_t s);
pet_status launch_svrg_anchor_finish(const float *B, int ns, long long plane, int nz,
                                     const float *sens, float *qtil, cudaStream_t s);
pet_status launch_saga_finish(const void *table, int table_dtype, int ns, long long plane, int nz,
                              const float *f0, const float *sens, float *qbar, float *d,
                              cudaStream_t s);
pet_status launch_table_mean(const void *table, int table_dtype, int ns, long long plane, float *mean,
                             cudaStream_t s);
pet_status launch_precond(const float *f0, const float *sens, int ns, long long plane, int nz,
                          float *d, cudaStream_t s);

}  // namespace petvr
