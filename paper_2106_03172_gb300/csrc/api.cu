// Host side of the C ABI declared in include/petvr.h: argument checking,
// geometry tables, object lifetime and the per-update launch sequences.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <thread>

#include "petvr_internal.cuh"

namespace petvr {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_error;

pet_status set_error(pet_status code, const std::string &msg) {
    t_error = msg;
    return code;
}

namespace {
struct ProfileRecord {
    int kind;
    cudaEvent_t a, b;
};
std::atomic<bool> g_profile{false};
std::mutex g_profile_mu;
std::vector<ProfileRecord> g_profile_records;
}  // namespace

bool profiling_enabled() { return g_profile.load(std::memory_order_relaxed); }

ProfileScope::ProfileScope(int k, cudaStream_t s) : kind(k), stream(s) {
    if (!g_profile.load(std::memory_order_relaxed)) return;
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaGetLastError();
        ev[0] = ev[1] = nullptr;
        return;
    }
    cudaEventRecord(ev[0], stream);
}

ProfileScope::~ProfileScope() {
    if (!ev[0]) return;
    cudaEventRecord(ev[1], stream);
    std::lock_guard<std::mutex> lk(g_profile_mu);
    g_profile_records.push_back({kind, ev[0], ev[1]});
}

bool use_pdl() {
    static const bool on = [] {
        const char *e = std::getenv("PETVR_NO_PDL");
        return !(e && e[0] && e[0] != '0');
    }();
    return on && !profiling_enabled();
}

pet_status check_launch(const char *what) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PET_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return PET_OK;
}

namespace {

constexpr long long kMaxElems = (1LL << 31) - 1;

template <typename T>
pet_status dalloc(T **p, size_t count, const char *what) {
    *p = nullptr;
    if (count == 0) return PET_OK;
    const cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? PET_ERR_OOM : PET_ERR_CUDA,
                         std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
    }
    return PET_OK;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

pet_status cuda_ok(cudaError_t e, const char *what) {
    if (e != cudaSuccess) return set_error(PET_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return PET_OK;
}

#define PET_TRY(expr)                          \
    do {                                       \
        const pet_status _st = (expr);         \
        if (_st != PET_OK) return _st;         \
    } while (0)

double snap(double v) {
    if (std::fabs(v) < 1e-12) return 0.0;
    if (std::fabs(v - 1.0) < 1e-12) return 1.0;
    if (std::fabs(v + 1.0) < 1e-12) return -1.0;
    return v;
}

int max_sub_rays(const pet_plan *pl) { return pl->max_sub_views * pl->nb; }

// Sinogram entries per (view, bin): slices of a stack, or ring pairs.
int sino_inner(const pet_plan *pl) { return pl->ring ? pl->pairs : pl->nz; }

// Blocks (log-likelihood partials) of a full-data forward pass, an upper
// bound over the launch shapes launch_forward may pick (multi-ring launches
// widen their band chunks up to 32 when the grid would be small).
int full_forward_blocks(const pet_plan *pl) {
    if (pl->ring) return forward_blocks(pl->na * pl->nb, 1, 32);
    return forward_blocks(pl->M, pl->nz, choose_group(pl));
}

FwdArgs fwd_args(const pet_plan *pl, const float *img, int subset, bool natural) {
    FwdArgs a{};
    a.views = pl->d_views;
    a.uc = pl->d_uc;
    a.order = natural ? pl->d_natural : pl->d_order;
    if (subset < 0) {
        a.v_begin = 0;
        a.v_end = pl->na;
    } else {
        a.v_begin = pl->sub_off[subset];
        a.v_end = pl->sub_off[subset + 1];
    }
    a.nx = pl->nx;
    a.ny = pl->ny;
    a.nz = sino_inner(pl);
    a.nb = pl->nb;
    a.layers = pl->layers;
    a.lz = pl->d_lz;
    a.img = img;
    return a;
}

BackArgs back_args(const pet_plan *pl, const float *r, int subset, bool natural) {
    BackArgs a{};
    a.views = pl->d_views;
    a.uc = pl->d_uc;
    a.order = natural ? pl->d_natural : pl->d_order;
    a.sub_off = natural ? pl->d_all_off : pl->d_sub_off;
    a.t0 = subset < 0 ? 0 : subset;
    a.r_view0 = subset < 0 ? 0 : pl->sub_off[subset];
    a.nx = pl->nx;
    a.ny = pl->ny;
    a.nz = pl->ring ? pl->layers : pl->nz;
    a.nb = pl->nb;
    a.ns = pl->ns;
    a.axial = pl->ring;
    a.pairs = pl->pairs;
    a.lz = pl->d_lz;
    a.r = r;
    a.sens_t = pl->d_sens_t;
    a.sens = pl->d_sens;
    a.run = pl->back_run;
    return a;
}

long long plane_of(const pet_plan *pl) { return (long long)pl->N * pl->nz; }

// Subset-t ratio r_t = g_t / (A_t f + w_t) into `ratio` (compact).
pet_status ratio_subset(const pet_problem *p, const float *f, int t, float *ratio, cudaStream_t s) {
    const pet_plan *pl = p->plan;
    FwdArgs a = fwd_args(pl, f, t, false);
    const long long off = (long long)pl->sub_off[t] * pl->nb * sino_inner(pl);
    a.g = p->d_g + off;
    a.w = p->d_w ? p->d_w + off : nullptr;
    a.w_scalar = p->w_scalar;
    a.out = ratio;
    a.status = p->d_status;
    return launch_forward(a, FWD_RATIO, false, choose_group(pl), s, nullptr);
}

// Full-data ratio in subset-major order into `ratio` (M * nz).
pet_status ratio_all(const pet_problem *p, const float *f, float *ratio, cudaStream_t s) {
    const pet_plan *pl = p->plan;
    FwdArgs a = fwd_args(pl, f, -1, false);
    a.g = p->d_g;
    a.w = p->d_w;
    a.w_scalar = p->w_scalar;
    a.out = ratio;
    a.status = p->d_status;
    return launch_forward(a, FWD_RATIO, false, full_group(pl), s, nullptr);
}

// n_iter updates with the iterate ping-ponging between the caller's image and
// `alt`, arranged so that the last update writes the caller's image.
template <class Step>
pet_status pingpong(float *user, float *alt, long long plane, int n_iter, cudaStream_t s, Step &&step) {
    if (n_iter <= 0) return PET_OK;
    float *a = user, *b = alt;
    if (n_iter % 2 == 1) {
        PET_TRY(cuda_ok(cudaMemcpyAsync(alt, user, (size_t)plane * sizeof(float), cudaMemcpyDeviceToDevice, s),
                        "cudaMemcpyAsync"));
        a = alt;
        b = user;
    }
    for (int i = 0; i < n_iter; ++i) {
        const float *in = (i % 2 == 0) ? a : b;
        float *out = (i % 2 == 0) ? b : a;
        PET_TRY(step(i, in, out));
    }
    return PET_OK;
}

pet_status check_seq(const pet_plan *pl, const int32_t *seq, int32_t n_iter) {
    if (n_iter < 0) return set_error(PET_ERR_INVALID, "n_iter must be >= 0");
    if (n_iter > 0 && !seq) return set_error(PET_ERR_INVALID, "null subset sequence");
    for (int i = 0; i < n_iter; ++i)
        if (seq[i] < 0 || seq[i] >= pl->ns)
            return set_error(PET_ERR_INVALID, "subset index out of range at position " + std::to_string(i));
    return PET_OK;
}

pet_status read_status(const pet_problem *p, cudaStream_t s) {
    int h = 0;
    PET_TRY(cuda_ok(cudaMemcpyAsync(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy"));
    PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    if (h != 0) {
        PET_TRY(cuda_ok(cudaMemsetAsync(p->d_status, 0, sizeof(int), s), "status reset"));
        return set_error((pet_status)h, "device reported a numeric error (nonpositive expected count)");
    }
    return PET_OK;
}

// Device bytes pet_state_create allocates for `algo` on plan pl.
size_t state_bytes(const pet_plan *pl, int algo, int table_dtype) {
    const size_t Nz = (size_t)pl->N * pl->nz, Mz = (size_t)pl->M * pl->nz;
    const size_t n_part = (size_t)full_forward_blocks(pl) + (Nz + 255) / 256;
    const size_t table_bytes = (size_t)pl->ns * Nz * (table_dtype == PET_TABLE_BF16 ? 2 : 4);
    size_t bytes = Nz * 4 + (size_t)max_sub_rays(pl) * sino_inner(pl) * 4 + n_part * 8;
    if (algo == PET_ALGO_SVREM) bytes += 3 * Nz * 4 + (size_t)pl->ns * Nz * 4 + Mz * 4;
    if (algo == PET_ALGO_SVRG) bytes += 2 * Nz * 4 + (size_t)pl->ns * Nz * 4 + Mz * 4;
    if (algo == PET_ALGO_SAGA) bytes += 2 * Nz * 4 + table_bytes;
    if (algo == PET_ALGO_SEM) bytes += Nz * 4 + Mz * 4;
    if (algo == PET_ALGO_SAGAEM) bytes += 2 * Nz * 4 + (size_t)pl->ns * Nz * 4;
    return bytes;
}

// (Re)initialise an allocated state at its current image: update counter,
// SVREM statistic flag, SAGA table/mean/preconditioner, SVRG preconditioner.
pet_status state_init(pet_state *st, cudaStream_t s) {
    const pet_problem *p = st->prob;
    const pet_plan *pl = p->plan;
    const long long Nz = plane_of(pl);
    st->k = 0;
    st->s_hat_ready = false;
    if (st->algo == PET_ALGO_SVRG) return launch_precond(st->img, pl->d_sens, pl->ns, Nz, pl->nz, st->d, s);
    if (st->algo == PET_ALGO_SAGAEM) {
        // table T_t = tau_t(f^(0)) for all t, its mean, and s_hat = mean = s(f^(0))
        PET_TRY(ratio_all(p, st->img, p->d_ratio, s));
        BackArgs b = back_args(pl, p->d_ratio, -1, false);
        b.t0 = 0;
        b.r_view0 = 0;
        b.f = st->img;
        b.table = st->table;
        PET_TRY(launch_back(b, EPI_SAGAEM_INIT, PET_TABLE_FP32, pl->ns, s, pl->max_sub_views));
        PET_TRY(launch_table_mean(st->table, PET_TABLE_FP32, pl->ns, Nz, st->qbar, s));
        return cuda_ok(cudaMemcpyAsync(st->s_hat, st->qbar, (size_t)Nz * 4, cudaMemcpyDeviceToDevice, s),
                       "statistic copy");
    }
    if (st->algo != PET_ALGO_SAGA) return PET_OK;
    // table q_t = grad Phi_t(f^(0)) for all t, then qbar and d
    PET_TRY(ratio_all(p, st->img, p->d_ratio, s));
    BackArgs b = back_args(pl, p->d_ratio, -1, false);
    b.t0 = 0;
    b.r_view0 = 0;
    b.f = st->img;
    b.beta = p->pen.beta;
    b.pot = p->pen.potential;
    b.delta = p->pen.delta;
    b.table = st->table;
    PET_TRY(launch_back(b, EPI_SAGA_INIT, st->table_dtype, pl->ns, s, pl->max_sub_views));
    return launch_saga_finish(st->table, st->table_dtype, pl->ns, Nz, pl->nz, st->img, pl->d_sens, st->qbar, st->d,
                              s);
}

// The warm start (a constant image, then one unpenalised OSEM epoch in cyclic
// subset order) into d_img, with `alt` (the image's size), `ratio` (a subset's
// rays) and `sums` (nz + 1 doubles; null: the problem's) as scratch: a state's
// own buffers let states of one problem warm-start on several streams at once.
pet_status warm_start_into(const pet_problem *p, float *d_img, float *alt, float *ratio, double *sums,
                           cudaStream_t s) {
    const pet_plan *pl = p->plan;
    PET_TRY(launch_uniform_image(p, d_img, s, sums));
    return pingpong(d_img, alt, plane_of(pl), pl->ns, s, [&](int i, const float *in, float *outp) {
        PET_TRY(ratio_subset(p, in, i, ratio, s));
        BackArgs b = back_args(pl, ratio, i, false);
        b.f = in;
        b.f_out = outp;
        b.beta = 0.0f;
        return launch_back(b, EPI_OSEM, PET_TABLE_FP32, 1, s, pl->max_sub_views);
    });
}

// Phi, L, R of d_img into d_phi (3 doubles), using `part` as block-partial scratch.
// With `ratio_out`, the same forward pass also writes the full-data ratio
// g / (A f + w) there (subset-major, as ratio_all): the sums are the ones
// ratio_all forms, so the ratios are bit-identical to a separate ratio_all.
pet_status objective_enqueue(const pet_problem *p, const float *d_img, double *d_phi, double *part,
                             cudaStream_t s, float *ratio_out = nullptr) {
    const pet_plan *pl = p->plan;
    FwdArgs a = fwd_args(pl, d_img, -1, false);
    a.g = p->d_g;
    a.w = p->d_w;
    a.w_scalar = p->w_scalar;
    a.ll_partials = part;
    a.out = ratio_out;
    a.status = p->d_status;
    int n_ll = 0;
    PET_TRY(launch_forward(a, ratio_out ? FWD_RATIO : FWD_NONE, true, full_group(pl), s, &n_ll));
    return launch_objective_finish(p, d_img, n_ll, part, d_phi, s);
}

}  // namespace
}  // namespace petvr

using namespace petvr;

extern "C" {

const char *pet_last_error(void) { return t_error.c_str(); }

uint64_t pet_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

pet_status pet_profile_enable(int32_t on) {
    g_profile.store(on != 0);
    return PET_OK;
}

pet_status pet_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_profile_mu);
    for (auto &r : g_profile_records) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_profile_records.clear();
    return PET_OK;
}

pet_status pet_profile_read(int32_t kind, int64_t *h_launches, double *h_total_ms) {
    if (!h_launches || !h_total_ms) return set_error(PET_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(g_profile_mu);
    int64_t n = 0;
    double total = 0.0;
    for (auto &r : g_profile_records) {
        if (r.kind != kind) continue;
        PET_TRY(cuda_ok(cudaEventSynchronize(r.b), "cudaEventSynchronize"));
        float ms = 0.0f;
        PET_TRY(cuda_ok(cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime"));
        total += ms;
        ++n;
    }
    *h_launches = n;
    *h_total_ms = total;
    return PET_OK;
}

void pet_plan_destroy(pet_plan *pl) {
    if (!pl) return;
    dfree(pl->d_views);
    dfree(pl->d_uc);
    dfree(pl->d_order);
    dfree(pl->d_natural);
    dfree(pl->d_sub_off);
    dfree(pl->d_all_off);
    dfree(pl->d_sens_t);
    dfree(pl->d_sens);
    dfree(pl->d_lz);
    delete pl;
}

pet_status pet_plan_create(const pet_geometry *g, const pet_subsets *sub, pet_plan **out) {
    if (!g || !sub || !out) return set_error(PET_ERR_INVALID, "null argument");
    *out = nullptr;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->n_angles < 1 || g->n_bins < 1)
        return set_error(PET_ERR_INVALID, "geometry sizes must be >= 1");
    if (g->nx > 16384 || g->ny > 16384) return set_error(PET_ERR_INVALID, "nx, ny must be <= 16384");
    if (g->n_angles > 1024) return set_error(PET_ERR_INVALID, "n_angles must be <= 1024");
    if (!(g->pixel_mm > 0.0) || !std::isfinite(g->pixel_mm) || !std::isfinite(g->bin_mm))
        return set_error(PET_ERR_INVALID, "pixel_mm must be positive and finite");
    if (sub->scheme != 0) return set_error(PET_ERR_INVALID, "only the interleaved subset scheme (0) exists");
    if (sub->n_subsets < 1 || sub->n_subsets > g->n_angles)
        return set_error(PET_ERR_INVALID, "need 1 <= n_subsets <= n_angles");
    const bool ring = g->n_rings > 0;
    const double ds_chk = g->bin_mm > 0.0 ? g->bin_mm : g->pixel_mm;
    if (ring) {
        if (g->n_rings > 4) return set_error(PET_ERR_INVALID, "n_rings must be <= 4");
        if (!(g->slice_mm > 0.0) || !std::isfinite(g->slice_mm) || !(g->ring_mm >= 0.0) ||
            !std::isfinite(g->ring_mm) || !std::isfinite(g->radius_mm))
            return set_error(PET_ERR_INVALID, "multi-ring geometry needs slice_mm > 0 and finite ring_mm >= 0");
        if (!(g->radius_mm > 0.5 * (g->n_bins - 1) * ds_chk))
            return set_error(PET_ERR_INVALID, "radius_mm must exceed every bin offset |s_j|");
    }
    const int pairs = ring ? g->n_rings * g->n_rings : 1;
    const long long N = (long long)g->nx * g->ny * (ring ? g->nz : 1);
    const long long M = (long long)g->n_angles * g->n_bins * pairs;
    if (N * (ring ? 1 : g->nz) > kMaxElems || M * (ring ? 1 : g->nz) > kMaxElems)
        return set_error(PET_ERR_INVALID, "image or sinogram larger than 2^31 - 1 elements");

    pet_plan *pl = new (std::nothrow) pet_plan();
    if (!pl) return set_error(PET_ERR_OOM, "host allocation failed");
    pl->geom = *g;
    pl->nx = g->nx;
    pl->ny = g->ny;
    pl->nz = ring ? 1 : g->nz;
    pl->ring = ring ? 1 : 0;
    pl->layers = ring ? g->nz : 1;
    pl->pairs = pairs;
    pl->na = g->n_angles;
    pl->nb = g->n_bins;
    pl->ns = sub->n_subsets;
    pl->N = (int)N;
    pl->M = (int)M;
    cudaGetDevice(&pl->device);
    const double d = g->pixel_mm;
    const double ds = g->bin_mm > 0.0 ? g->bin_mm : d;

    // per-view parameters and per-ray centred minor offsets (FP64 -> FP32)
    std::vector<ViewParams> views(pl->na);
    const long long R = (long long)pl->na * pl->nb;        // rays of the transaxial geometry
    std::vector<float2> uc((size_t)R);
    // multi-ring: per line, zeta(kc) = zc + zs kc in layer units and sqrt(1 + kappa^2)
    std::vector<float4> lz(ring ? (size_t)M : 0);
    const double z_min = -0.5 * g->nz * g->slice_mm;
    for (int i = 0; i < pl->na; ++i) {
        const double th = (double)i * M_PI / (double)pl->na;
        const double c = snap(std::cos(th)), s = snap(std::sin(th));
        ViewParams vp{};
        vp.col = std::fabs(c) < std::fabs(s) ? 1 : 0;
        const double cm = vp.col ? s : c;          // direction cosine of the major axis
        const double cn = vp.col ? c : s;          // of the minor axis
        const int n_minor = vp.col ? pl->ny : pl->nx;
        const double du = -cn / cm;
        vp.du = (float)du;
        vp.du_lo = (float)(du - (double)vp.du);
        vp.L = (float)(d / std::fabs(cm));
        vp.Lm = cn != 0.0 ? (float)(d / std::fabs(cn)) : 0.0f;
        vp.K = (float)(ds / (cm * d));
        vp.invK = (float)(cm * d / ds);
        vp.inv_du = cn != 0.0 ? (float)(-cm / cn) : 0.0f;
        const double off = (n_minor % 2) ? 0.5 : 0.0;
        for (int j = 0; j < pl->nb; ++j) {
            const double sj = ((double)j - 0.5 * (pl->nb - 1)) * ds;
            const double u = sj / (cm * d) + off;
            const double ui = std::nearbyint(u);
            uc[(size_t)i * pl->nb + j] = make_float2((float)ui, (float)(u - ui));
            if (j == 0) vp.uc0 = (float)u;
            if (!ring) continue;
            // transaxial arc length t(kc) = t0 + t1 kc along (-sin, cos) at centred major coordinate kc
            const double t0 = vp.col ? sj * c / s : -sj * s / c;
            const double t1 = vp.col ? -d / s : d / c;
            const double T = std::sqrt(g->radius_mm * g->radius_mm - sj * sj);
            for (int r1 = 0; r1 < g->n_rings; ++r1)
                for (int r2 = 0; r2 < g->n_rings; ++r2) {
                    const double z1 = (r1 - 0.5 * (g->n_rings - 1)) * g->ring_mm;
                    const double z2 = (r2 - 0.5 * (g->n_rings - 1)) * g->ring_mm;
                    const double kappa = (z2 - z1) / (2.0 * T);
                    const double zm = 0.5 * (z1 + z2);
                    lz[((size_t)i * pl->nb + j) * pairs + r1 * g->n_rings + r2] =
                        make_float4((float)((zm + kappa * t0 - z_min) / g->slice_mm),
                                    (float)(kappa * t1 / g->slice_mm), (float)std::sqrt(1.0 + kappa * kappa), 0.0f);
                }
        }
        views[i] = vp;
    }
    // angle-interleaved subsets: view i -> subset i mod ns
    pl->sub_off.assign(pl->ns + 1, 0);
    for (int t = 0; t < pl->ns; ++t) {
        for (int i = t; i < pl->na; i += pl->ns) pl->order.push_back(i);
        pl->sub_off[t + 1] = (int)pl->order.size();
        pl->max_sub_views = std::max(pl->max_sub_views, pl->sub_off[t + 1] - pl->sub_off[t]);
    }
    std::vector<int> natural(pl->na);
    for (int i = 0; i < pl->na; ++i) natural[i] = i;
    const int all_off[2] = {0, pl->na};

    pet_status st = PET_OK;
    float *ones = nullptr;
    auto fail = [&](pet_status e) {
        dfree(ones);
        pet_plan_destroy(pl);
        return e;
    };
    if ((st = dalloc(&pl->d_views, pl->na, "views")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_uc, (size_t)R, "uc")) != PET_OK) return fail(st);
    if (ring && (st = dalloc(&pl->d_lz, (size_t)M, "lz")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_order, pl->na, "order")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_natural, pl->na, "natural")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_sub_off, pl->ns + 1, "sub_off")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_all_off, 2, "all_off")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_sens_t, (size_t)pl->ns * N, "sens_t")) != PET_OK) return fail(st);
    if ((st = dalloc(&pl->d_sens, (size_t)N, "sens")) != PET_OK) return fail(st);
    if ((st = dalloc(&ones, (size_t)M, "ones")) != PET_OK) return fail(st);
    cudaError_t e = cudaSuccess;
    e = cudaMemcpy(pl->d_views, views.data(), sizeof(ViewParams) * pl->na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_uc, uc.data(), sizeof(float2) * R, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ring) e = cudaMemcpy(pl->d_lz, lz.data(), sizeof(float4) * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_order, pl->order.data(), sizeof(int) * pl->na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_natural, natural.data(), sizeof(int) * pl->na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_sub_off, pl->sub_off.data(), sizeof(int) * (pl->ns + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_all_off, all_off, sizeof(int) * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_ok(e, "table upload"));
    {
        std::vector<float> h1((size_t)M, 1.0f);
        e = cudaMemcpy(ones, h1.data(), sizeof(float) * M, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_ok(e, "ones upload"));
    }
    // sens_t = A_t^T 1 for every subset (one slice of a stack: the geometry is shared
    // by all slices; every voxel of a multi-ring volume)
    BackArgs b = back_args(pl, ones, -1, false);
    if (!ring) b.nz = 1;
    b.t0 = 0;
    b.r_view0 = 0;
    b.out = pl->d_sens_t;
    if ((st = launch_back(b, EPI_ANCHOR, PET_TABLE_FP32, pl->ns, 0, pl->max_sub_views)) != PET_OK) return fail(st);
    if ((st = launch_sum_sens(pl->d_sens_t, pl->d_sens, pl->ns, pl->N, 0)) != PET_OK) return fail(st);
    // nonzeros per subset, counted with the projector's own geometry
    {
        unsigned long long *d_cnt = nullptr;
        if ((st = dalloc(&d_cnt, (size_t)pl->ns, "nnz")) != PET_OK) return fail(st);
        e = cudaMemset(d_cnt, 0, sizeof(unsigned long long) * pl->ns);
        for (int t = 0; t < pl->ns && e == cudaSuccess && st == PET_OK; ++t) {
            FwdArgs a = fwd_args(pl, nullptr, t, false);
            if (!ring) a.nz = 1;
            st = launch_count_nnz(a, d_cnt + t, 0);
        }
        std::vector<unsigned long long> h((size_t)pl->ns, 0);
        if (e == cudaSuccess && st == PET_OK)
            e = cudaMemcpy(h.data(), d_cnt, sizeof(unsigned long long) * pl->ns, cudaMemcpyDeviceToHost);
        dfree(d_cnt);
        if (st != PET_OK) return fail(st);
        if (e != cudaSuccess) return fail(cuda_ok(e, "nnz count"));
        pl->nnz.assign(h.begin(), h.end());
    }
    e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return fail(cuda_ok(e, "plan sensitivity"));
    dfree(ones);
    *out = pl;
    return PET_OK;
}

pet_status pet_plan_subset_views(const pet_plan *pl, int32_t t, int32_t *h_n) {
    if (!pl || !h_n) return set_error(PET_ERR_INVALID, "null argument");
    if (t < -1 || t >= pl->ns) return set_error(PET_ERR_INVALID, "subset out of range");
    *h_n = t < 0 ? pl->na : pl->sub_off[t + 1] - pl->sub_off[t];
    return PET_OK;
}

pet_status pet_plan_nnz(const pet_plan *pl, int32_t t, int64_t *h_nnz) {
    if (!pl || !h_nnz) return set_error(PET_ERR_INVALID, "null argument");
    if (t < -1 || t >= pl->ns) return set_error(PET_ERR_INVALID, "subset out of range");
    long long n = 0;
    for (int i = 0; i < pl->ns; ++i)
        if (t < 0 || i == t) n += pl->nnz[i];
    *h_nnz = n;
    return PET_OK;
}

pet_status pet_plan_bytes(const pet_plan *pl, size_t *h_bytes) {
    if (!pl || !h_bytes) return set_error(PET_ERR_INVALID, "null argument");
    *h_bytes = sizeof(ViewParams) * pl->na + sizeof(float2) * (size_t)pl->M + sizeof(int) * (2 * (size_t)pl->na + pl->ns + 3) +
               sizeof(float) * ((size_t)pl->ns + 1) * pl->N;
    return PET_OK;
}

pet_status pet_problem_bytes(const pet_plan *pl, int32_t has_bg, size_t *h_bytes) {
    if (!pl || !h_bytes) return set_error(PET_ERR_INVALID, "null argument");
    const size_t Mz = (size_t)pl->M * pl->nz, Nz = (size_t)pl->N * pl->nz;
    const size_t n_part = (size_t)full_forward_blocks(pl) + (Nz + 255) / 256;
    *h_bytes = sizeof(float) * (Mz * (has_bg ? 3 : 2) + Nz) + sizeof(double) * (n_part + pl->nz + 8) + sizeof(int);
    return PET_OK;
}

pet_status pet_plan_state_bytes(const pet_plan *pl, int32_t algo, int32_t table_dtype, size_t *h_bytes) {
    if (!pl || !h_bytes) return set_error(PET_ERR_INVALID, "null argument");
    if (algo < PET_ALGO_OSEM || algo > PET_ALGO_SAGAEM) return set_error(PET_ERR_INVALID, "unknown algorithm");
    *h_bytes = state_bytes(pl, algo, table_dtype);
    return PET_OK;
}

pet_status pet_plan_set_tuning(pet_plan *pl, int32_t fwd_chunks, int32_t back_run) {
    if (!pl) return set_error(PET_ERR_INVALID, "null plan");
    if (fwd_chunks != 0 && fwd_chunks != 8 && fwd_chunks != 16 && fwd_chunks != 32)
        return set_error(PET_ERR_INVALID, "fwd_chunks must be 0 (default), 8, 16 or 32");
    if (back_run != 4 && back_run != 8) return set_error(PET_ERR_INVALID, "back_run must be 4 or 8");
    pl->fwd_chunks = fwd_chunks;
    pl->back_run = back_run;
    return PET_OK;
}

pet_status pet_plan_get_tuning(const pet_plan *pl, int32_t *h_fwd_chunks, int32_t *h_back_run) {
    if (!pl || !h_fwd_chunks || !h_back_run) return set_error(PET_ERR_INVALID, "null argument");
    *h_fwd_chunks = choose_group(pl);
    *h_back_run = pl->back_run;
    return PET_OK;
}

pet_status pet_plan_autotune(pet_plan *pl, int32_t *h_fwd_chunks, int32_t *h_back_run) {
    if (!pl) return set_error(PET_ERR_INVALID, "null plan");
    if (pl->nz == 1 && !pl->ring) {
        const size_t N = (size_t)pl->N, R = (size_t)max_sub_rays(pl);
        float *img = nullptr, *sino = nullptr, *out = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        pet_status st = PET_OK;
        auto cleanup = [&]() {
            dfree(img);
            dfree(sino);
            dfree(out);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (s) cudaStreamDestroy(s);
        };
        if ((st = dalloc(&img, N, "tune image")) != PET_OK || (st = dalloc(&sino, R, "tune sinogram")) != PET_OK ||
            (st = dalloc(&out, N, "tune image")) != PET_OK) {
            cleanup();
            return st;
        }
        std::vector<float> ones(std::max(N, R), 1.0f);
        cudaError_t e = cudaMemcpy(img, ones.data(), N * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(sino, ones.data(), R * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_ok(e, "autotune set-up");
        }
        // time `reps` passes over every subset of one projector, best of 3
        auto time_pass = [&](bool forward, float *best_ms) -> pet_status {
            float best = 1e30f;
            for (int trial = 0; trial < 4; ++trial) {
                PET_TRY(cuda_ok(cudaEventRecord(e0, s), "event"));
                for (int t = 0; t < pl->ns; ++t) {
                    if (forward) {
                        FwdArgs a = fwd_args(pl, img, t, false);
                        a.out = sino;
                        PET_TRY(launch_forward(a, FWD_YHAT, false, choose_group(pl), s, nullptr));
                    } else {
                        BackArgs b = back_args(pl, sino, t, false);
                        b.out = out;
                        PET_TRY(launch_back(b, EPI_PLAIN, PET_TABLE_FP32, 1, s, pl->max_sub_views));
                    }
                }
                PET_TRY(cuda_ok(cudaEventRecord(e1, s), "event"));
                PET_TRY(cuda_ok(cudaEventSynchronize(e1), "event sync"));
                float ms = 0.0f;
                PET_TRY(cuda_ok(cudaEventElapsedTime(&ms, e0, e1), "event time"));
                if (trial > 0) best = std::min(best, ms);   // trial 0 warms up
            }
            *best_ms = best;
            return PET_OK;
        };
        int best_c = choose_group(pl), best_r = pl->back_run;
        float best_ms = 1e30f;
        for (int c : {8, 16, 32}) {
            pl->fwd_chunks = c;
            float ms = 0.0f;
            if ((st = time_pass(true, &ms)) != PET_OK) break;
            if (ms < best_ms) best_ms = ms, best_c = c;
        }
        pl->fwd_chunks = best_c;
        best_ms = 1e30f;
        // 4-pixel runs need blocks twice as wide as 8-pixel runs, so fewer fit
        // beside other streams' kernels and the all-subset launches (anchors,
        // table fills) slow down: measured on the 256^2 four-stream step, run 4
        // took its subset back projections from 9.6 to 10.4 us and its anchor
        // from 47 to 93 us, and the step from 28.2 to 40.6 ms.  Timed alone the
        // two are close, so run 4 is taken only when it is clearly faster.
        for (int r : {8, 4}) {
            if (st != PET_OK) break;
            pl->back_run = r;
            float ms = 0.0f;
            if ((st = time_pass(false, &ms)) != PET_OK) break;
            if (ms < best_ms * (r == 4 ? 0.85f : 1.0f)) best_ms = ms, best_r = r;
        }
        pl->back_run = best_r;
        cleanup();
        if (st != PET_OK) return st;
    }
    if (h_fwd_chunks) *h_fwd_chunks = choose_group(pl);
    if (h_back_run) *h_back_run = pl->back_run;
    return PET_OK;
}

pet_status pet_plan_sensitivity(const pet_plan *pl, int32_t t, float *d_out, void *stream) {
    if (!pl || !d_out) return set_error(PET_ERR_INVALID, "null argument");
    if (t < -1 || t >= pl->ns) return set_error(PET_ERR_INVALID, "subset out of range");
    const float *src = t < 0 ? pl->d_sens : pl->d_sens_t + (size_t)t * pl->N;
    return cuda_ok(cudaMemcpyAsync(d_out, src, sizeof(float) * pl->N, cudaMemcpyDeviceToDevice,
                                   (cudaStream_t)stream),
                   "sensitivity copy");
}

pet_status pet_forward(const pet_plan *pl, const float *d_img, const float *d_bg, float bg, int32_t subset,
                       float *d_sino, void *stream) {
    if (!pl || !d_img || !d_sino) return set_error(PET_ERR_INVALID, "null argument");
    if (subset < -1 || subset >= pl->ns) return set_error(PET_ERR_INVALID, "subset out of range");
    if (!std::isfinite(bg)) return set_error(PET_ERR_INVALID, "background must be finite");
    FwdArgs a = fwd_args(pl, d_img, subset, subset < 0);
    a.w = d_bg;
    a.w_scalar = bg;
    a.out = d_sino;
    return launch_forward(a, FWD_YHAT, false, subset < 0 ? full_group(pl) : choose_group(pl), (cudaStream_t)stream,
                          nullptr);
}

pet_status pet_back(const pet_plan *pl, const float *d_sino, int32_t subset, float *d_img, void *stream) {
    if (!pl || !d_img || !d_sino) return set_error(PET_ERR_INVALID, "null argument");
    if (subset < -1 || subset >= pl->ns) return set_error(PET_ERR_INVALID, "subset out of range");
    BackArgs b = back_args(pl, d_sino, subset, subset < 0);
    b.out = d_img;
    return launch_back(b, EPI_PLAIN, PET_TABLE_FP32, 1, (cudaStream_t)stream,
                       subset < 0 ? pl->na : pl->max_sub_views);
}

void pet_problem_destroy(pet_problem *p) {
    if (!p) return;
    dfree(p->d_g);
    dfree(p->d_w);
    dfree(p->d_ratio);
    dfree(p->d_alt);
    dfree(p->d_part);
    dfree(p->d_scalar);
    dfree(p->d_status);
    delete p;
}

pet_status pet_problem_create(const pet_plan *pl, const float *d_counts, const float *d_bg, float bg,
                              const pet_penalty *pen, pet_problem **out, void *stream) {
    if (!pl || !d_counts || !pen || !out) return set_error(PET_ERR_INVALID, "null argument");
    *out = nullptr;
    if (pen->potential < PET_POT_QUADRATIC || pen->potential > PET_POT_HYPERBOLA)
        return set_error(PET_ERR_INVALID, "unknown potential");
    if (pen->potential != PET_POT_QUADRATIC && !(pen->delta > 0.0f && std::isfinite(pen->delta)))
        return set_error(PET_ERR_INVALID, "delta must be positive and finite");
    if (!(pen->beta >= 0.0f) || !std::isfinite(pen->beta)) return set_error(PET_ERR_INVALID, "beta must be >= 0");
    if (!std::isfinite(bg)) return set_error(PET_ERR_INVALID, "background must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    pet_problem *p = new (std::nothrow) pet_problem();
    if (!p) return set_error(PET_ERR_OOM, "host allocation failed");
    p->plan = pl;
    p->pen = *pen;
    p->w_scalar = bg;
    const size_t Mz = (size_t)pl->M * pl->nz, Nz = (size_t)pl->N * pl->nz;
    p->n_part = full_forward_blocks(pl) + (int)((Nz + 255) / 256);
    pet_status st;
    auto fail = [&](pet_status e) {
        pet_problem_destroy(p);
        return e;
    };
    if ((st = dalloc(&p->d_g, Mz, "counts")) != PET_OK) return fail(st);
    if (d_bg && (st = dalloc(&p->d_w, Mz, "background")) != PET_OK) return fail(st);
    if ((st = dalloc(&p->d_ratio, Mz, "ratio")) != PET_OK) return fail(st);
    if ((st = dalloc(&p->d_alt, Nz, "alt image")) != PET_OK) return fail(st);
    if ((st = dalloc(&p->d_part, (size_t)p->n_part, "partials")) != PET_OK) return fail(st);
    if ((st = dalloc(&p->d_scalar, (size_t)pl->nz + 8, "scalars")) != PET_OK) return fail(st);
    if ((st = dalloc(&p->d_status, 1, "status")) != PET_OK) return fail(st);
    if ((st = cuda_ok(cudaMemsetAsync(p->d_status, 0, sizeof(int), s), "memset")) != PET_OK) return fail(st);
    if ((st = launch_permute_sino(d_counts, p->d_g, pl->d_order, pl->na, pl->nb, sino_inner(pl), s)) != PET_OK)
        return fail(st);
    if (d_bg && (st = launch_permute_sino(d_bg, p->d_w, pl->d_order, pl->na, pl->nb, sino_inner(pl), s)) != PET_OK)
        return fail(st);
    *out = p;
    return PET_OK;
}

pet_status pet_problem_update(pet_problem *p, const float *d_counts, const float *d_bg, float bg, void *stream) {
    if (!p || !d_counts) return set_error(PET_ERR_INVALID, "null argument");
    if ((d_bg != nullptr) != (p->d_w != nullptr))
        return set_error(PET_ERR_INVALID, "background kind differs from the one the problem was created with");
    if (!std::isfinite(bg)) return set_error(PET_ERR_INVALID, "background must be finite");
    const pet_plan *pl = p->plan;
    cudaStream_t s = (cudaStream_t)stream;
    if (bg != p->w_scalar) {        // counts are read through pointers; the scalar is captured by value
        p->w_scalar = bg;
        ++p->version;
    }
    PET_TRY(launch_permute_sino(d_counts, p->d_g, pl->d_order, pl->na, pl->nb, sino_inner(pl), s));
    if (d_bg) PET_TRY(launch_permute_sino(d_bg, p->d_w, pl->d_order, pl->na, pl->nb, sino_inner(pl), s));
    return PET_OK;
}

pet_status pet_warm_start(const pet_problem *p, float *d_img, void *stream) {
    if (!p || !d_img) return set_error(PET_ERR_INVALID, "null argument");
    return warm_start_into(p, d_img, p->d_alt, p->d_ratio, nullptr, (cudaStream_t)stream);
}

pet_status pet_objective_async(const pet_problem *p, const float *d_img, double *d_phi, void *stream) {
    if (!p || !d_img || !d_phi) return set_error(PET_ERR_INVALID, "null argument");
    return objective_enqueue(p, d_img, d_phi, p->d_part, (cudaStream_t)stream);
}

pet_status pet_objective(const pet_problem *p, const float *d_img, double *h_phi, void *stream) {
    if (!p || !d_img || !h_phi) return set_error(PET_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    PET_TRY(pet_objective_async(p, d_img, p->d_scalar, stream));
    PET_TRY(cuda_ok(cudaMemcpyAsync(h_phi, p->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s), "phi copy"));
    return read_status(p, s);
}

pet_status pet_state_destroy(pet_state *st) {
    if (!st) return PET_OK;
    dfree(st->alt);
    dfree(st->ratio);
    dfree(st->ratio_full);
    dfree(st->s_hat);
    dfree(st->f_anc);
    dfree(st->s_anc);
    dfree(st->B);
    dfree(st->d);
    dfree(st->qbar);
    dfree(st->qtil);
    if (st->table) cudaFree(st->table);
    dfree(st->d_seq);
    dfree(st->d_alpha);
    dfree(st->d_part);
    for (auto &g : st->graphs) cudaGraphExecDestroy(g.exec);
    if (st->cap) cudaStreamDestroy(st->cap);
    delete st;
    return PET_OK;
}

pet_status pet_state_create(const pet_problem *p, int32_t algo, int32_t table_dtype, float *d_img,
                            size_t *bytes_needed, pet_state **out, void *stream) {
    if (!p) return set_error(PET_ERR_INVALID, "null problem");
    if (algo < PET_ALGO_OSEM || algo > PET_ALGO_SAGAEM) return set_error(PET_ERR_INVALID, "unknown algorithm");
    if (algo == PET_ALGO_SAGAEM && table_dtype != PET_TABLE_FP32)
        return set_error(PET_ERR_INVALID, "the SAGA-EM statistic table is FP32");
    if (table_dtype != PET_TABLE_FP32 && table_dtype != PET_TABLE_BF16)
        return set_error(PET_ERR_INVALID, "unknown table dtype");
    const pet_plan *pl = p->plan;
    const size_t Nz = (size_t)pl->N * pl->nz;
    const size_t table_bytes = (size_t)pl->ns * Nz * (table_dtype == PET_TABLE_BF16 ? 2 : 4);
    const size_t bytes = state_bytes(pl, algo, table_dtype);
    if (bytes_needed) *bytes_needed = bytes;
    if (!out) return PET_OK;
    *out = nullptr;
    if (!d_img) return set_error(PET_ERR_INVALID, "null image");
    cudaStream_t s = (cudaStream_t)stream;
    pet_state *st = new (std::nothrow) pet_state();
    if (!st) return set_error(PET_ERR_OOM, "host allocation failed");
    st->prob = p;
    st->algo = algo;
    st->table_dtype = table_dtype;
    st->img = d_img;
    st->bytes = bytes;
    pet_status e;
    auto fail = [&](pet_status code) {
        pet_state_destroy(st);
        return code;
    };
    const size_t Mz = (size_t)pl->M * pl->nz;
    if ((e = dalloc(&st->alt, Nz, "alt")) != PET_OK) return fail(e);
    st->n_part = p->n_part;
    if ((e = dalloc(&st->d_part, (size_t)st->n_part, "objective partials")) != PET_OK) return fail(e);
    if ((e = dalloc(&st->ratio, (size_t)max_sub_rays(pl) * sino_inner(pl), "ratio")) != PET_OK) return fail(e);
    if (algo == PET_ALGO_SVREM) {
        if ((e = dalloc(&st->s_hat, Nz, "s_hat")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->f_anc, Nz, "f_anc")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->s_anc, Nz, "s_anc")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->B, (size_t)pl->ns * Nz, "B")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->ratio_full, Mz, "full ratio")) != PET_OK) return fail(e);
    } else if (algo == PET_ALGO_SEM) {
        if ((e = dalloc(&st->s_hat, Nz, "s_hat")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->ratio_full, Mz, "full ratio")) != PET_OK) return fail(e);
    } else if (algo == PET_ALGO_SAGAEM) {
        if ((e = dalloc(&st->s_hat, Nz, "s_hat")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->qbar, Nz, "table mean")) != PET_OK) return fail(e);
        const cudaError_t ce = cudaMalloc(&st->table, (size_t)pl->ns * Nz * 4);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            st->table = nullptr;
            return fail(set_error(PET_ERR_OOM, "cudaMalloc SAGA-EM table"));
        }
    } else if (algo == PET_ALGO_SVRG) {
        if ((e = dalloc(&st->d, Nz, "d")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->qtil, Nz, "q_tilde")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->B, (size_t)pl->ns * Nz, "B")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->ratio_full, Mz, "full ratio")) != PET_OK) return fail(e);
    } else if (algo == PET_ALGO_SAGA) {
        if ((e = dalloc(&st->d, Nz, "d")) != PET_OK) return fail(e);
        if ((e = dalloc(&st->qbar, Nz, "qbar")) != PET_OK) return fail(e);
        const cudaError_t ce = cudaMalloc(&st->table, table_bytes);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            st->table = nullptr;
            return fail(set_error(PET_ERR_OOM, "cudaMalloc SAGA table"));
        }
    }
    if ((e = state_init(st, s)) != PET_OK) return fail(e);
    *out = st;
    return PET_OK;
}

}  // extern "C"

namespace {

// Anchor pass at f: B_t = A_t^T r_t(f) for every t, into st->B, one forward
// launch over all rays (skipped when `ratios_ready`: ratio_full already holds
// r(f), written by the objective of f) and one back launch over all subsets
// (grid.y = t).
pet_status anchor_pass(pet_state *st, const float *f, float *ratio_full, cudaStream_t s, bool ratios_ready = false) {
    const pet_problem *p = st->prob;
    const pet_plan *pl = p->plan;
    if (!ratios_ready) PET_TRY(ratio_all(p, f, ratio_full, s));
    BackArgs b = back_args(pl, ratio_full, -1, false);
    b.t0 = 0;
    b.r_view0 = 0;
    b.out = st->B;
    return launch_back(b, EPI_ANCHOR, PET_TABLE_FP32, pl->ns, s, pl->max_sub_views);
}

// One update on subset *t_dev (device-resident index) from `in` to `outp`.
pet_status enqueue_update(pet_state *st, int algo, const int *t_dev, const float *alpha_dev, const float *in,
                          float *outp, cudaStream_t s) {
    const pet_problem *p = st->prob;
    const pet_plan *pl = p->plan;
    FwdArgs a = fwd_args(pl, in, -1, false);
    a.t_dev = t_dev;
    a.sub_off = pl->d_sub_off;
    a.g = p->d_g;
    a.w = p->d_w;
    a.w_scalar = p->w_scalar;
    a.out = st->ratio;
    a.status = p->d_status;
    PET_TRY(launch_forward(a, FWD_RATIO, false, choose_group(pl), s, nullptr, max_sub_rays(pl)));
    BackArgs b = back_args(pl, st->ratio, 0, false);
    b.t_dev = t_dev;
    b.f = in;
    b.f_out = outp;
    b.beta = p->pen.beta;
    b.pot = p->pen.potential;
    b.delta = p->pen.delta;
    b.alpha_dev = alpha_dev;
    int epi = EPI_OSEM;
    if (algo == PET_ALGO_SVREM) {
        epi = EPI_SVREM;
        b.s_hat = st->s_hat;
        b.f_anc = st->f_anc;
        b.s_anc = st->s_anc;
        b.B = st->B;
    } else if (algo == PET_ALGO_SAGA) {
        epi = EPI_SAGA;
        b.d = st->precond == PET_PRECOND_ITERATE ? nullptr : st->d;
        b.table = st->table;
        b.qbar = st->qbar;
    } else if (algo == PET_ALGO_SVRG) {
        epi = EPI_SVRG;
        b.d = st->precond == PET_PRECOND_ITERATE ? nullptr : st->d;
        b.B = st->B;
        b.qtil = st->qtil;
    } else if (algo == PET_ALGO_SGA) {
        epi = EPI_SGA;
    } else if (algo == PET_ALGO_SEM) {
        epi = EPI_SEM;
        b.s_hat = st->s_hat;
    } else if (algo == PET_ALGO_SAGAEM) {
        epi = EPI_SAGAEM;
        b.s_hat = st->s_hat;
        b.table = st->table;
        b.qbar = st->qbar;
    }
    return launch_back(b, epi, st->table_dtype, 1, s, pl->max_sub_views);
}

// SEM start: s_hat = f . A^T(g / (A f + w)), the full statistic at f (one pass).
pet_status sem_init(pet_state *st, const float *f, cudaStream_t s) {
    const pet_problem *p = st->prob;
    const pet_plan *pl = p->plan;
    PET_TRY(ratio_all(p, f, st->ratio_full, s));
    BackArgs b = back_args(pl, st->ratio_full, -1, false);
    b.sub_off = pl->d_all_off;            // every view, in the subset-major order of the ratio
    b.t0 = 0;
    b.r_view0 = 0;
    b.f = f;
    b.s_hat = st->s_hat;
    return launch_back(b, EPI_SEM_INIT, PET_TABLE_FP32, 1, s, pl->na);
}

// The whole launch sequence of n_iter updates (anchors where `anchors[i]`),
// on stream s.  With every > 0, the objective of the iterate after update i
// goes to d_phi[3 j .. 3 j + 2], j = (i + 1) / every - 1, whenever every
// divides i + 1.  An objective whose iterate is the next update's anchor
// (SVREM, SVRG) writes that anchor's ratios in the same forward pass, and the
// anchor pass then starts from its back projection.
pet_status enqueue_epoch(pet_state *st, int algo, int32_t n_iter, const std::vector<uint8_t> &anchors,
                         cudaStream_t s, int every = 0, double *d_phi = nullptr) {
    const pet_plan *pl = st->prob->plan;
    const long long plane = plane_of(pl);
    const bool anchored = algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG;
    bool ratios_ready = false;      // st->ratio_full holds the ratios of the next update's input
    return pingpong(st->img, st->alt, plane, n_iter, s, [&](int i, const float *in, float *outp) {
        if (anchors[i] && algo == PET_ALGO_SVREM) {
            PET_TRY(anchor_pass(st, in, st->ratio_full, s, ratios_ready));
            PET_TRY(launch_svrem_anchor_finish(st->B, pl->ns, plane, pl->nz, in, st->f_anc, st->s_anc, st->s_hat,
                                               !st->s_hat_ready, s));
            st->s_hat_ready = true;
        } else if (anchors[i] && algo == PET_ALGO_SVRG) {
            PET_TRY(anchor_pass(st, in, st->ratio_full, s, ratios_ready));
            PET_TRY(launch_svrg_anchor_finish(st->B, pl->ns, plane, pl->nz, pl->d_sens, st->qtil, s));
        }
        ratios_ready = false;
        if (algo == PET_ALGO_SEM && !st->s_hat_ready) {
            PET_TRY(sem_init(st, in, s));
            st->s_hat_ready = true;
        }
        PET_TRY(enqueue_update(st, algo, st->d_seq + i, st->d_alpha + i, in, outp, s));
        if (every > 0 && (i + 1) % every == 0) {
            const bool share = anchored && i + 1 < n_iter && anchors[i + 1];
            PET_TRY(objective_enqueue(st->prob, outp, d_phi + 3LL * ((i + 1) / every - 1), st->d_part, s,
                                      share ? st->ratio_full : nullptr));
            ratios_ready = share;
        }
        return PET_OK;
    });
}

bool use_graphs() {
    static const bool on = [] {
        const char *e = std::getenv("PETVR_NO_GRAPHS");
        return !(e && e[0] && e[0] != '0');
    }();
    return on;
}

// Executable graphs a state (or a batch) keeps: a caller that passes a new
// output buffer on every call (the buffer is a kernel argument, so part of
// the key) would otherwise grow the cache without bound.  The least recently
// launched graph is destroyed first; one still in flight is freed by the
// driver once its launch completes.
constexpr size_t kMaxGraphs = 64;

// Capture `enqueue` once on the state's private stream, cache the executable
// graph under `key`, and launch it on `s`.
template <class Enqueue>
pet_status run_graph(pet_state *st, const std::vector<int64_t> &key, cudaStream_t s, Enqueue &&enqueue) {
    if (st->prob && st->graph_version != st->prob->version) {
        // the problem's data changed since these were captured (kernel
        // arguments such as the scalar background are baked into a graph)
        for (auto &g : st->graphs) cudaGraphExecDestroy(g.exec);
        st->graphs.clear();
        st->graph_version = st->prob->version;
    }
    pet_state::Graph *hit = nullptr;
    for (auto &g : st->graphs)
        if (g.key == key) hit = &g;
    if (!hit) {
        if (!st->cap) PET_TRY(cuda_ok(cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking), "capture stream"));
        PET_TRY(cuda_ok(cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal), "begin capture"));
        const uint64_t before = g_launches.load();
        const pet_status est = enqueue(st->cap);
        // launches recorded into the graph are counted when the graph runs
        const uint64_t kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(st->cap, &graph);
        if (est != PET_OK) {
            if (graph) cudaGraphDestroy(graph);
            return est;
        }
        PET_TRY(cuda_ok(ce, "end capture"));
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        PET_TRY(cuda_ok(ie, "graph instantiate"));
        if (st->graphs.size() >= kMaxGraphs) {
            auto lru = st->graphs.begin();
            for (auto it = st->graphs.begin(); it != st->graphs.end(); ++it)
                if (it->last_use < lru->last_use) lru = it;
            cudaGraphExecDestroy(lru->exec);
            st->graphs.erase(lru);
        }
        st->graphs.push_back({key, exec, kernels, 0});
        hit = &st->graphs.back();
    }
    hit->last_use = ++st->graph_tick;
    PET_TRY(cuda_ok(cudaGraphLaunch(hit->exec, s), "graph launch"));
    g_launches.fetch_add(hit->kernels);
    return PET_OK;
}

pet_status epoch_common(pet_state *st, int algo, const int32_t *seq, int32_t n_iter, float alpha0, float decay,
                        int32_t eta, cudaStream_t s, int32_t every = 0, double *d_phi = nullptr) {
    if (!st) return set_error(PET_ERR_INVALID, "null state");
    if (st->algo != algo) return set_error(PET_ERR_STATE, "state was created for another algorithm");
    const pet_problem *p = st->prob;
    const pet_plan *pl = p->plan;
    PET_TRY(check_seq(pl, seq, n_iter));
    if (!std::isfinite(alpha0) || !std::isfinite(decay) || decay < 0.0f)
        return set_error(PET_ERR_INVALID, "alpha must be finite and decay >= 0");
    if ((algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG) && eta < 1)
        return set_error(PET_ERR_INVALID, "eta must be >= 1");
    if (n_iter == 0) return PET_OK;
    if (n_iter > st->seq_cap) {
        int *grown = nullptr;
        float *grown_a = nullptr;
        PET_TRY(dalloc(&grown, (size_t)n_iter, "subset sequence"));
        if (dalloc(&grown_a, (size_t)n_iter, "step sizes") != PET_OK) {
            dfree(grown);
            return PET_ERR_OOM;
        }
        // the old buffers may still be read by enqueued work: release them after the stream drains
        if (st->d_seq) {
            PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
            dfree(st->d_seq);
            dfree(st->d_alpha);
        }
        st->d_seq = grown;
        st->d_alpha = grown_a;
        st->seq_cap = n_iter;
        for (auto &g : st->graphs) cudaGraphExecDestroy(g.exec);
        st->graphs.clear();
    }
    std::vector<float> alphas((size_t)n_iter);
    for (int i = 0; i < n_iter; ++i) alphas[i] = (float)((double)alpha0 / ((double)decay * (double)(st->k + i) + 1.0));
    PET_TRY(cuda_ok(cudaMemcpyAsync(st->d_seq, seq, sizeof(int32_t) * n_iter, cudaMemcpyHostToDevice, s),
                    "subset sequence copy"));
    PET_TRY(cuda_ok(cudaMemcpyAsync(st->d_alpha, alphas.data(), sizeof(float) * n_iter, cudaMemcpyHostToDevice, s),
                    "step size copy"));
    std::vector<uint8_t> anchors((size_t)n_iter, 0);
    if (algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG)
        for (int i = 0; i < n_iter; ++i) anchors[i] = ((st->k + i) % ((long long)eta * pl->ns) == 0) ? 1 : 0;
    pet_status rc;
    // a first SVREM anchor / SEM start also initialises s_hat: that call is enqueued directly
    const bool first = (algo == PET_ALGO_SVREM || algo == PET_ALGO_SEM) && !st->s_hat_ready;
    if (!use_graphs() || profiling_enabled() || first) {
        rc = enqueue_epoch(st, algo, n_iter, anchors, s, every, d_phi);
    } else {
        std::vector<int64_t> key = {n_iter, eta};
        if (every > 0) {                    // objectives inside: a separate graph per output buffer
            key.push_back(-2);
            key.push_back(every);
            key.push_back((int64_t)(intptr_t)d_phi);
        }
        for (int i = 0; i < n_iter; ++i)
            if (anchors[i]) key.push_back(i);
        rc = run_graph(st, key, s,
                       [&](cudaStream_t cs) { return enqueue_epoch(st, algo, n_iter, anchors, cs, every, d_phi); });
    }
    if (rc == PET_OK) st->k += n_iter;
    return rc;
}

}  // namespace

extern "C" {

pet_status pet_osem_epoch(pet_state *st, const int32_t *seq, int32_t n_iter, void *stream) {
    return epoch_common(st, PET_ALGO_OSEM, seq, n_iter, 0.0f, 0.0f, 1, (cudaStream_t)stream);
}

pet_status pet_svrem_epoch(pet_state *st, float alpha, int32_t eta, const int32_t *seq, int32_t n_iter,
                           void *stream) {
    return epoch_common(st, PET_ALGO_SVREM, seq, n_iter, alpha, 0.0f, eta, (cudaStream_t)stream);
}

pet_status pet_saga_epoch(pet_state *st, float alpha, const int32_t *seq, int32_t n_iter, void *stream) {
    return epoch_common(st, PET_ALGO_SAGA, seq, n_iter, alpha, 0.0f, 1, (cudaStream_t)stream);
}

pet_status pet_svrg_epoch(pet_state *st, float alpha, int32_t eta, const int32_t *seq, int32_t n_iter,
                          void *stream) {
    return epoch_common(st, PET_ALGO_SVRG, seq, n_iter, alpha, 0.0f, eta, (cudaStream_t)stream);
}

pet_status pet_sga_epoch(pet_state *st, float alpha0, float decay, const int32_t *seq, int32_t n_iter,
                         void *stream) {
    return epoch_common(st, PET_ALGO_SGA, seq, n_iter, alpha0, decay, 1, (cudaStream_t)stream);
}

pet_status pet_sem_epoch(pet_state *st, float alpha0, float decay, const int32_t *seq, int32_t n_iter,
                         void *stream) {
    return epoch_common(st, PET_ALGO_SEM, seq, n_iter, alpha0, decay, 1, (cudaStream_t)stream);
}

pet_status pet_sagaem_epoch(pet_state *st, float alpha, const int32_t *seq, int32_t n_iter, void *stream) {
    return epoch_common(st, PET_ALGO_SAGAEM, seq, n_iter, alpha, 0.0f, 1, (cudaStream_t)stream);
}

pet_status pet_state_run(pet_state *st, const int32_t *seq, int32_t n_iter, float alpha, float decay, int32_t eta,
                         int32_t objective_every, double *d_phi, void *stream) {
    if (!st) return set_error(PET_ERR_INVALID, "null state");
    if (objective_every < 0) return set_error(PET_ERR_INVALID, "objective_every must be >= 0");
    if (objective_every > 0 && !d_phi) return set_error(PET_ERR_INVALID, "null d_phi with objective_every > 0");
    const int algo = st->algo;
    // the epoch calls' conventions: OSEM takes no step size, only SVREM and SVRG an anchor period
    const bool stepped = algo != PET_ALGO_OSEM;
    return epoch_common(st, algo, seq, n_iter, stepped ? alpha : 0.0f, stepped ? decay : 0.0f,
                        (algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG) ? eta : 1, (cudaStream_t)stream,
                        objective_every, d_phi);
}

pet_status pet_state_objective_async(pet_state *st, double *d_phi, void *stream) {
    if (!st || !d_phi) return set_error(PET_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!use_graphs() || profiling_enabled())
        return objective_enqueue(st->prob, st->img, d_phi, st->d_part, s);
    const std::vector<int64_t> key = {-1, (int64_t)(intptr_t)d_phi};
    return run_graph(st, key, s, [&](cudaStream_t cs) {
        return objective_enqueue(st->prob, st->img, d_phi, st->d_part, cs);
    });
}

// ---- executor: many reconstructions to an objective gap ------------------------

}  // extern "C"

namespace petvr {
namespace {

// One reconstruction of the executor: the state it runs on (a worker's, or
// its own), its subset sequence (max_epochs * N_s indices), its step and its
// reference optimum.
struct GapJob {
    pet_state *st;
    const int32_t *seq;
    float a0, dc;
    int eta;
    double phi_star;
};

// The step conventions of the epoch calls for a state's algorithm, checked.
pet_status job_steps(int algo, float alpha, float decay, int32_t eta, GapJob &j) {
    const bool stepped = algo != PET_ALGO_OSEM;
    j.a0 = stepped ? alpha : 0.0f;
    j.dc = stepped ? decay : 0.0f;
    j.eta = (algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG) ? eta : 1;
    if (!std::isfinite(j.a0) || !std::isfinite(j.dc) || j.dc < 0.0f)
        return set_error(PET_ERR_INVALID, "alpha must be finite and decay >= 0");
    if (j.eta < 1) return set_error(PET_ERR_INVALID, "eta must be >= 1");
    return PET_OK;
}

// Runs the jobs to the gap on n_slots streams of its own.  Worker-pool mode
// (workers non-null): slot w runs its jobs on workers[w] and copies each
// job's final image to results (when non-null); otherwise each job runs on
// its own state, which keeps the final image.  The host loop: a job starts
// with the warm start (the state's own scratch) and the state's reset, then
// one epoch and its objective at a time, each read back to pinned host memory
// behind an event; the host polls the events, and after each objective either
// launches the job's next epoch or records the job and starts the next one on
// that slot.  Resets that fill a SAGA / SAGA-EM table go through their
// problem's full-data ratio buffer, so those of one problem are chained by an
// event.  Synchronising; the slots start after the work enqueued on `caller`.
// With arrival_s, job j starts only once arrival_s[j] seconds have passed
// since the call (h_start_ms / h_done_ms: times since the call).  With the
// hooks, the caller owns the jobs' states: `acquire` gives job j its state
// (ok = false: not now, the job waits at the head of the queue) just before
// it starts on stream `s`; `release` runs at the job's end, after its last
// objective was read.
using AcquireFn = std::function<pet_status(int, cudaStream_t, bool &)>;
using ReleaseFn = std::function<pet_status(int, cudaStream_t)>;

pet_status drive_to_gap(std::vector<GapJob> &jobs, int n_slots, pet_state *const *workers, float *results,
                        int max_epochs, double gap, int32_t *h_epochs, double *h_gap, double *h_ms,
                        cudaStream_t caller, const double *arrival_s = nullptr, double *h_start_ms = nullptr,
                        double *h_done_ms = nullptr, const AcquireFn *acquire = nullptr,
                        const ReleaseFn *release = nullptr) {
    using clock = std::chrono::steady_clock;
    const int n_jobs = (int)jobs.size();
    const clock::time_point t_call = clock::now();
    auto since_call_ms = [&](clock::time_point t) {
        return std::chrono::duration<double, std::milli>(t - t_call).count();
    };
    // arrival_s: job j may start only once arrival_s[j] seconds have passed since the call (nondecreasing)
    auto arrived = [&](int j) { return !arrival_s || since_call_ms(clock::now()) >= 1e3 * arrival_s[j]; };
    struct Slot {
        pet_state *worker = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        double *d_phi = nullptr;
        int job = -1, epoch = 0;
        clock::time_point t0;
    };
    std::vector<Slot> slots((size_t)n_slots);
    std::vector<std::pair<const pet_problem *, cudaEvent_t>> chains;    // SAGA / SAGA-EM resets per problem
    std::vector<const pet_problem *> chained;                           // problems whose chain has an event
    double *h_phi = nullptr, *d_phi = nullptr;
    cudaEvent_t entry = nullptr;
    pet_status rc = PET_OK;
    auto cleanup = [&]() {
        for (Slot &sl : slots) {
            if (sl.s) cudaStreamSynchronize(sl.s);
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.s) cudaStreamDestroy(sl.s);
        }
        for (auto &c : chains) cudaEventDestroy(c.second);
        if (entry) cudaEventDestroy(entry);
        if (h_phi) cudaFreeHost(h_phi);
        dfree(d_phi);
    };
    auto fail = [&](pet_status st) {
        cleanup();
        return st;
    };
    if ((rc = cuda_ok(cudaMallocHost(&h_phi, sizeof(double) * 3 * n_slots), "pinned objectives")) != PET_OK)
        return fail(rc);
    if ((rc = dalloc(&d_phi, (size_t)3 * n_slots, "objectives")) != PET_OK) return fail(rc);
    if ((rc = cuda_ok(cudaEventCreateWithFlags(&entry, cudaEventDisableTiming), "event")) != PET_OK) return fail(rc);
    if ((rc = cuda_ok(cudaEventRecord(entry, caller), "event record")) != PET_OK) return fail(rc);
    for (int w = 0; w < n_slots; ++w) {
        Slot &sl = slots[(size_t)w];
        sl.worker = workers ? workers[w] : nullptr;
        sl.d_phi = d_phi + 3 * w;
        if ((rc = cuda_ok(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking), "worker stream")) != PET_OK ||
            (rc = cuda_ok(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming), "event")) != PET_OK ||
            (rc = cuda_ok(cudaStreamWaitEvent(sl.s, entry, 0), "stream wait")) != PET_OK)
            return fail(rc);
    }
    auto launch_epoch = [&](int w) -> pet_status {
        Slot &sl = slots[(size_t)w];
        const GapJob &j = jobs[(size_t)sl.job];
        const int ns = j.st->prob->plan->ns;
        PET_TRY(epoch_common(j.st, j.st->algo, j.seq + (long long)sl.epoch * ns, ns, j.a0, j.dc, j.eta, sl.s));
        PET_TRY(pet_state_objective_async(j.st, sl.d_phi, sl.s));
        PET_TRY(cuda_ok(cudaMemcpyAsync(h_phi + 3 * w, sl.d_phi, sizeof(double) * 3, cudaMemcpyDeviceToHost, sl.s),
                        "objective copy"));
        return cuda_ok(cudaEventRecord(sl.ev, sl.s), "event record");
    };
    int next = 0;
    auto start_job = [&](int w) -> pet_status {
        Slot &sl = slots[(size_t)w];
        sl.job = next++;
        sl.epoch = 0;
        sl.t0 = clock::now();
        if (h_start_ms) h_start_ms[sl.job] = since_call_ms(sl.t0);
        GapJob &j = jobs[(size_t)sl.job];
        if (sl.worker) j.st = sl.worker;
        pet_state *st = j.st;
        const pet_problem *p = st->prob;
        PET_TRY(warm_start_into(p, st->img, st->alt, st->ratio, st->d_part, sl.s));
        const bool shared = st->algo == PET_ALGO_SAGA || st->algo == PET_ALGO_SAGAEM;
        cudaEvent_t chain = nullptr;
        if (shared) {
            for (auto &c : chains)
                if (c.first == p) chain = c.second;
            if (!chain) {
                PET_TRY(cuda_ok(cudaEventCreateWithFlags(&chain, cudaEventDisableTiming), "event"));
                chains.push_back({p, chain});
            } else {
                PET_TRY(cuda_ok(cudaStreamWaitEvent(sl.s, chain, 0), "stream wait"));
            }
        }
        PET_TRY(state_init(st, sl.s));
        if (shared) PET_TRY(cuda_ok(cudaEventRecord(chain, sl.s), "event record"));
        return launch_epoch(w);
    };
    int active = 0;
    while (active > 0 || next < n_jobs) {
        bool progressed = false;
        // free slots take the jobs that have arrived, in order
        for (int w = 0; w < n_slots && next < n_jobs; ++w) {
            if (slots[(size_t)w].job >= 0 || !arrived(next)) continue;
            if (acquire) {
                bool ok = false;
                if ((rc = (*acquire)(next, slots[(size_t)w].s, ok)) != PET_OK) return fail(rc);
                if (!ok) break;
            }
            if ((rc = start_job(w)) != PET_OK) return fail(rc);
            ++active;
            progressed = true;
        }
        for (int w = 0; w < n_slots; ++w) {
            Slot &sl = slots[(size_t)w];
            if (sl.job < 0) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            if ((rc = cuda_ok(q, "event query")) != PET_OK) return fail(rc);
            progressed = true;
            ++sl.epoch;
            const GapJob &j = jobs[(size_t)sl.job];
            const double g = (j.phi_star - h_phi[3 * w]) / std::fabs(j.phi_star);
            if (g <= gap || sl.epoch >= max_epochs || !std::isfinite(g)) {
                const clock::time_point t_done = clock::now();
                h_epochs[sl.job] = sl.epoch;
                h_gap[sl.job] = g;
                h_ms[sl.job] = std::chrono::duration<double, std::milli>(t_done - sl.t0).count();
                if (h_done_ms) h_done_ms[sl.job] = since_call_ms(t_done);
                if (sl.worker && results) {
                    const long long plane = plane_of(j.st->prob->plan);
                    if ((rc = cuda_ok(cudaMemcpyAsync(results + (long long)sl.job * plane, j.st->img,
                                                      sizeof(float) * (size_t)plane, cudaMemcpyDeviceToDevice, sl.s),
                                      "result copy")) != PET_OK)
                        return fail(rc);
                }
                if (release && (rc = (*release)(sl.job, sl.s)) != PET_OK) return fail(rc);
                sl.job = -1;
                --active;
                if (!acquire && next < n_jobs && arrived(next)) {
                    if ((rc = start_job(w)) != PET_OK) return fail(rc);
                    ++active;
                }
            } else if ((rc = launch_epoch(w)) != PET_OK) {
                return fail(rc);
            }
        }
        if (!progressed) {
            // nothing running and the next job far off: sleep until shortly before it arrives
            const double ahead_ms = (active == 0 && next < n_jobs && arrival_s)
                                        ? 1e3 * arrival_s[next] - since_call_ms(clock::now()) : 0.0;
            if (ahead_ms > 2.0)
                std::this_thread::sleep_for(std::chrono::microseconds((long long)(1e3 * (ahead_ms - 1.0))));
            else
                std::this_thread::yield();
        }
    }
    cleanup();
    if (acquire) return PET_OK;    // the caller owns (and checks) the jobs' problems
    // numeric errors latched by any job's problem
    for (const GapJob &j : jobs) {
        bool seen = false;
        for (const GapJob &i : jobs) {
            if (&i == &j) break;
            if (i.st->prob == j.st->prob) seen = true;
        }
        if (!seen) PET_TRY(read_status(j.st->prob, caller));
    }
    return PET_OK;
}

pet_status check_gap_args(int32_t n_jobs, int32_t max_epochs, double gap, const void *seqs, const int32_t *h_epochs,
                          const double *h_gap, const double *h_ms) {
    if (n_jobs < 0 || max_epochs < 1) return set_error(PET_ERR_INVALID, "n_jobs must be >= 0 and max_epochs >= 1");
    if (n_jobs > 0 && (!seqs || !h_epochs || !h_gap || !h_ms)) return set_error(PET_ERR_INVALID, "null argument");
    if (!std::isfinite(gap) || gap < 0.0) return set_error(PET_ERR_INVALID, "gap must be finite and >= 0");
    return PET_OK;
}

pet_status check_job_seq(const pet_plan *pl, const int32_t *seq, long long n, long long job) {
    for (long long i = 0; i < n; ++i)
        if (seq[i] < 0 || seq[i] >= pl->ns)
            return set_error(PET_ERR_INVALID, "subset index out of range in job " + std::to_string(job) +
                                                  " at position " + std::to_string(i));
    return PET_OK;
}

}  // namespace
}  // namespace petvr

extern "C" {

pet_status pet_run_to_gap(pet_state *const *workers, int32_t n_workers, int32_t n_jobs, const int32_t *h_seqs,
                          int32_t max_epochs, float alpha, float decay, int32_t eta, double phi_star, double gap,
                          float *d_results, int32_t *h_epochs, double *h_gap, double *h_ms, void *stream) {
    if (!workers || n_workers < 1) return set_error(PET_ERR_INVALID, "need at least one worker state");
    PET_TRY(check_gap_args(n_jobs, max_epochs, gap, h_seqs, h_epochs, h_gap, h_ms));
    if (!std::isfinite(phi_star) || phi_star == 0.0)
        return set_error(PET_ERR_INVALID, "phi_star must be finite and nonzero");
    for (int w = 0; w < n_workers; ++w) {
        if (!workers[w]) return set_error(PET_ERR_INVALID, "null worker state");
        if (workers[w]->prob != workers[0]->prob || workers[w]->algo != workers[0]->algo)
            return set_error(PET_ERR_INVALID, "worker states must share one problem and one algorithm");
        for (int v = 0; v < w; ++v)
            if (workers[v] == workers[w] || workers[v]->img == workers[w]->img)
                return set_error(PET_ERR_INVALID, "worker states must be distinct, with distinct images");
    }
    const pet_plan *pl = workers[0]->prob->plan;
    GapJob proto{nullptr, nullptr, 0.0f, 0.0f, 1, phi_star};
    PET_TRY(job_steps(workers[0]->algo, alpha, decay, eta, proto));
    const long long per_job = (long long)max_epochs * pl->ns;
    for (int j = 0; j < n_jobs; ++j) PET_TRY(check_job_seq(pl, h_seqs + (long long)j * per_job, per_job, j));
    if (n_jobs == 0) return PET_OK;
    std::vector<GapJob> jobs((size_t)n_jobs, proto);
    for (int j = 0; j < n_jobs; ++j) jobs[(size_t)j].seq = h_seqs + (long long)j * per_job;
    return drive_to_gap(jobs, std::min(n_workers, n_jobs), workers, d_results, max_epochs, gap, h_epochs, h_gap,
                        h_ms, (cudaStream_t)stream);
}

pet_status pet_run_jobs_to_gap(pet_state *const *states, const int32_t *const *h_seqs, const float *h_alpha,
                               const float *h_decay, const int32_t *h_eta, const double *h_phi_star, int32_t n_jobs,
                               int32_t n_streams, int32_t max_epochs, double gap, int32_t *h_epochs, double *h_gap,
                               double *h_ms, void *stream) {
    PET_TRY(check_gap_args(n_jobs, max_epochs, gap, h_seqs, h_epochs, h_gap, h_ms));
    if (n_streams < 1) return set_error(PET_ERR_INVALID, "n_streams must be >= 1");
    if (n_jobs > 0 && (!states || !h_alpha || !h_decay || !h_eta || !h_phi_star))
        return set_error(PET_ERR_INVALID, "null argument");
    std::vector<GapJob> jobs((size_t)n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        if (!states[j] || !h_seqs[j]) return set_error(PET_ERR_INVALID, "null state or sequence of job " + std::to_string(j));
        if (!std::isfinite(h_phi_star[j]) || h_phi_star[j] == 0.0)
            return set_error(PET_ERR_INVALID, "phi_star of job " + std::to_string(j) + " must be finite and nonzero");
        for (int i = 0; i < j; ++i)
            if (states[i] == states[j] || states[i]->img == states[j]->img)
                return set_error(PET_ERR_INVALID, "jobs must have distinct states with distinct images");
        GapJob &g = jobs[(size_t)j];
        g.st = states[j];
        g.seq = h_seqs[j];
        g.phi_star = h_phi_star[j];
        PET_TRY(job_steps(states[j]->algo, h_alpha[j], h_decay[j], h_eta[j], g));
        const pet_plan *pl = states[j]->prob->plan;
        PET_TRY(check_job_seq(pl, h_seqs[j], (long long)max_epochs * pl->ns, j));
    }
    if (n_jobs == 0) return PET_OK;
    return drive_to_gap(jobs, std::min(n_streams, n_jobs), nullptr, nullptr, max_epochs, gap, h_epochs, h_gap, h_ms,
                        (cudaStream_t)stream);
}

pet_status pet_serve_jobs(pet_state *const *states, const int32_t *const *h_seqs, const float *h_alpha,
                          const float *h_decay, const int32_t *h_eta, const double *h_phi_star,
                          const double *h_arrival_s, int32_t n_jobs, int32_t n_streams, int32_t max_epochs, double gap,
                          int32_t *h_epochs, double *h_gap, double *h_start_ms, double *h_done_ms, void *stream) {
    if (n_jobs > 0 && (!h_arrival_s || !h_start_ms || !h_done_ms)) return set_error(PET_ERR_INVALID, "null argument");
    for (int j = 0; j < n_jobs; ++j)
        if (!std::isfinite(h_arrival_s[j]) || h_arrival_s[j] < 0.0 || (j > 0 && h_arrival_s[j] < h_arrival_s[j - 1]))
            return set_error(PET_ERR_INVALID, "arrival times must be finite, >= 0 and nondecreasing");
    std::vector<double> ms((size_t)std::max(1, (int)n_jobs));
    PET_TRY(check_gap_args(n_jobs, max_epochs, gap, h_seqs, h_epochs, h_gap, ms.data()));
    if (n_streams < 1) return set_error(PET_ERR_INVALID, "n_streams must be >= 1");
    if (n_jobs > 0 && (!states || !h_alpha || !h_decay || !h_eta || !h_phi_star))
        return set_error(PET_ERR_INVALID, "null argument");
    std::vector<GapJob> jobs((size_t)n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        if (!states[j] || !h_seqs[j]) return set_error(PET_ERR_INVALID, "null state or sequence of job " + std::to_string(j));
        if (!std::isfinite(h_phi_star[j]) || h_phi_star[j] == 0.0)
            return set_error(PET_ERR_INVALID, "phi_star of job " + std::to_string(j) + " must be finite and nonzero");
        for (int i = 0; i < j; ++i)
            if (states[i] == states[j] || states[i]->img == states[j]->img)
                return set_error(PET_ERR_INVALID, "jobs must have distinct states with distinct images");
        GapJob &g = jobs[(size_t)j];
        g.st = states[j];
        g.seq = h_seqs[j];
        g.phi_star = h_phi_star[j];
        PET_TRY(job_steps(states[j]->algo, h_alpha[j], h_decay[j], h_eta[j], g));
        const pet_plan *pl = states[j]->prob->plan;
        PET_TRY(check_job_seq(pl, h_seqs[j], (long long)max_epochs * pl->ns, j));
    }
    if (n_jobs == 0) return PET_OK;
    return drive_to_gap(jobs, std::min(n_streams, n_jobs), nullptr, nullptr, max_epochs, gap, h_epochs, h_gap,
                        ms.data(), (cudaStream_t)stream, h_arrival_s, h_start_ms, h_done_ms);
}

pet_status pet_serve_requests(const pet_request *reqs, int32_t n, int32_t n_streams, size_t budget_bytes,
                              int32_t max_epochs, double gap, int32_t *h_epochs, double *h_gap, double *h_start_ms,
                              double *h_done_ms, pet_serve_stats *stats, void *stream) {
    std::vector<double> ms((size_t)std::max(1, (int)n));
    PET_TRY(check_gap_args(n, max_epochs, gap, reqs, h_epochs, h_gap, ms.data()));
    if (n_streams < 1) return set_error(PET_ERR_INVALID, "n_streams must be >= 1");
    if (n > 0 && (!h_start_ms || !h_done_ms || !stats)) return set_error(PET_ERR_INVALID, "null argument");
    std::vector<GapJob> jobs((size_t)n);
    std::vector<size_t> need((size_t)n);
    for (int j = 0; j < n; ++j) {
        const pet_request &r = reqs[j];
        const std::string at = " of request " + std::to_string(j);
        if (!r.plan || !r.h_counts || !r.h_seq) return set_error(PET_ERR_INVALID, "null plan, counts or sequence" + at);
        if (r.algo < PET_ALGO_OSEM || r.algo > PET_ALGO_SAGAEM) return set_error(PET_ERR_INVALID, "unknown algorithm" + at);
        if (r.table_dtype != PET_TABLE_FP32 && r.table_dtype != PET_TABLE_BF16)
            return set_error(PET_ERR_INVALID, "unknown table type" + at);
        if (!std::isfinite(r.bg)) return set_error(PET_ERR_INVALID, "background must be finite" + at);
        if (!std::isfinite(r.phi_star) || r.phi_star == 0.0)
            return set_error(PET_ERR_INVALID, "phi_star must be finite and nonzero" + at);
        if (!std::isfinite(r.arrival_s) || r.arrival_s < 0.0 || (j > 0 && r.arrival_s < reqs[j - 1].arrival_s))
            return set_error(PET_ERR_INVALID, "arrival times must be finite, >= 0 and nondecreasing");
        GapJob &g = jobs[(size_t)j];
        g.st = nullptr;
        g.seq = r.h_seq;
        g.phi_star = r.phi_star;
        PET_TRY(job_steps(r.algo, r.alpha, r.decay, r.eta, g));
        PET_TRY(check_job_seq(r.plan, r.h_seq, (long long)max_epochs * r.plan->ns, j));
        size_t pb = 0, sb = 0;
        PET_TRY(pet_problem_bytes(r.plan, 0, &pb));
        PET_TRY(pet_plan_state_bytes(r.plan, r.algo, r.table_dtype, &sb));
        need[(size_t)j] = pb + sb + sizeof(float) * ((size_t)r.plan->M * sino_inner(r.plan) + (size_t)plane_of(r.plan));
        if (need[(size_t)j] > budget_bytes) return set_error(PET_ERR_INVALID, "request larger than the budget" + at);
    }
    *stats = pet_serve_stats{};
    if (n == 0) return PET_OK;

    // the slot pool: a request's problem, state, image and counts staging, kept after the request for
    // the next one of the same plan, algorithm, table and penalty
    struct Pooled {
        const pet_request *key;
        pet_problem *p = nullptr;
        pet_state *st = nullptr;
        float *img = nullptr, *stage = nullptr;
        size_t bytes = 0;
        int job = -1;
        uint64_t used = 0;
    };
    std::vector<Pooled> pool;
    size_t used_bytes = 0;
    uint64_t tick = 0;
    int last_deferred = -1;
    auto same_kind = [](const pet_request &a, const pet_request &b) {
        return a.plan == b.plan && a.algo == b.algo && a.table_dtype == b.table_dtype &&
               a.penalty.potential == b.penalty.potential && a.penalty.beta == b.penalty.beta &&
               a.penalty.delta == b.penalty.delta;
    };
    auto destroy = [&](Pooled &q) -> pet_status {
        pet_status st = PET_OK;
        if (q.p) st = read_status(q.p, (cudaStream_t)stream);     // a numeric error latched by its requests
        pet_state_destroy(q.st);
        pet_problem_destroy(q.p);
        dfree(q.img);
        dfree(q.stage);
        used_bytes -= q.bytes;
        return st;
    };
    auto upload = [&](Pooled &q, const pet_request &r, cudaStream_t s) -> pet_status {
        const size_t count = (size_t)r.plan->M * sino_inner(r.plan);
        return cuda_ok(cudaMemcpyAsync(q.stage, r.h_counts, sizeof(float) * count, cudaMemcpyHostToDevice, s),
                       "counts upload");
    };
    const AcquireFn acquire = [&](int j, cudaStream_t s, bool &ok) -> pet_status {
        const pet_request &r = reqs[j];
        ok = false;
        for (Pooled &q : pool)
            if (q.job < 0 && same_kind(*q.key, r)) {
                PET_TRY(upload(q, r, s));
                PET_TRY(pet_problem_update(q.p, q.stage, nullptr, r.bg, s));
                q.job = j;
                q.used = ++tick;
                jobs[(size_t)j].st = q.st;
                ++stats->slots_reused;
                ok = true;
                return PET_OK;
            }
        // make room: free pooled slots, least recently used first
        while (used_bytes + need[(size_t)j] > budget_bytes) {
            Pooled *lru = nullptr;
            for (Pooled &q : pool)
                if (q.job < 0 && (!lru || q.used < lru->used)) lru = &q;
            if (!lru) break;
            const pet_status st = destroy(*lru);
            pool.erase(pool.begin() + (lru - pool.data()));
            ++stats->slots_evicted;
            PET_TRY(st);
        }
        if (used_bytes + need[(size_t)j] > budget_bytes) {          // wait for a running request to end
            if (last_deferred != j) ++stats->admissions_deferred;
            last_deferred = j;
            return PET_OK;
        }
        Pooled q;
        q.key = &r;
        q.bytes = need[(size_t)j];
        const pet_plan *pl = r.plan;
        pet_status st = dalloc(&q.stage, (size_t)pl->M * sino_inner(pl), "counts staging");
        if (st == PET_OK) st = dalloc(&q.img, (size_t)plane_of(pl), "image");
        // the state is made on a zero image (its job's warm start and reset come before any update)
        if (st == PET_OK)
            st = cuda_ok(cudaMemsetAsync(q.img, 0, sizeof(float) * (size_t)plane_of(pl), s), "image clear");
        if (st == PET_OK) st = upload(q, r, s);
        if (st == PET_OK) st = pet_problem_create(pl, q.stage, nullptr, r.bg, &r.penalty, &q.p, s);
        if (st == PET_OK) st = pet_state_create(q.p, r.algo, r.table_dtype, q.img, nullptr, &q.st, s);
        if (st != PET_OK) {
            pet_state_destroy(q.st);
            pet_problem_destroy(q.p);
            dfree(q.img);
            dfree(q.stage);
            return st;
        }
        q.job = j;
        q.used = ++tick;
        used_bytes += q.bytes;
        stats->peak_bytes = std::max(stats->peak_bytes, used_bytes);
        ++stats->slots_created;
        jobs[(size_t)j].st = q.st;
        pool.push_back(q);
        ok = true;
        return PET_OK;
    };
    const ReleaseFn release = [&](int j, cudaStream_t s) -> pet_status {
        for (Pooled &q : pool)
            if (q.job == j) {
                if (reqs[j].h_image) {
                    PET_TRY(cuda_ok(cudaMemcpyAsync(reqs[j].h_image, q.img, sizeof(float) * (size_t)plane_of(q.key->plan),
                                                    cudaMemcpyDeviceToHost, s), "image download"));
                    PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
                }
                q.job = -1;
                return PET_OK;
            }
        return set_error(PET_ERR_STATE, "released a request that holds no slot");
    };
    std::vector<double> arrivals((size_t)n);
    for (int j = 0; j < n; ++j) arrivals[(size_t)j] = reqs[j].arrival_s;
    pet_status rc = drive_to_gap(jobs, std::min((int)n_streams, (int)n), nullptr, nullptr, max_epochs, gap, h_epochs,
                                 h_gap, ms.data(), (cudaStream_t)stream, arrivals.data(), h_start_ms, h_done_ms,
                                 &acquire, &release);
    for (Pooled &q : pool) {
        const pet_status st = destroy(q);
        if (rc == PET_OK) rc = st;
    }
    return rc;
}

// ---- batches ------------------------------------------------------------------

pet_status pet_batch_destroy(pet_batch *b) {
    if (!b) return PET_OK;
    dfree(b->d_members);
    dfree(b->d_segs);
    dfree(b->d_claims);
    dfree(b->d_obj_segs);
    dfree(b->d_obj_claim);
    dfree(b->d_df);
    dfree(b->d_df_done);
    dfree(b->d_status);
    dfree(b->d_seqs);
    dfree(b->d_alphas);
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t sd : b->side) {
        cudaStreamSynchronize(sd);
        cudaStreamDestroy(sd);
    }
    for (cudaEvent_t e : b->side_ev) cudaEventDestroy(e);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    delete b;
    return PET_OK;
}

pet_status pet_batch_set_graphs(pet_batch *b, int32_t on) {
    if (!b) return set_error(PET_ERR_INVALID, "null batch");
    b->graphs_on = on != 0;
    return PET_OK;
}

pet_status pet_batch_set_mode(pet_batch *b, int32_t mode) {
    if (!b) return set_error(PET_ERR_INVALID, "null batch");
    if (mode != PET_BATCH_PHASES && mode != PET_BATCH_DATAFLOW && mode != PET_BATCH_STREAMS)
        return set_error(PET_ERR_INVALID, "unknown batch mode");
    b->mode = mode;
    return PET_OK;
}

pet_status pet_batch_set_wait_limit(pet_batch *b, int64_t polls) {
    if (!b) return set_error(PET_ERR_INVALID, "null batch");
    if (polls < 0) return set_error(PET_ERR_INVALID, "the wait limit must be >= 0");
    b->wait_limit = polls;
    // the limit is a kernel argument of the captured epochs
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    return PET_OK;
}

pet_status pet_batch_sync(pet_batch *b, void *stream) {
    if (!b) return set_error(PET_ERR_INVALID, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    PET_TRY(cuda_ok(cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy"));
    PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    if (h != 0) {
        PET_TRY(cuda_ok(cudaMemsetAsync(b->d_status, 0, sizeof(int), s), "status reset"));
        PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
        return set_error((pet_status)h, "a dependency wait of the batched epoch ran out (PET_ERR_TIMEOUT); the "
                                        "members' iterates are not valid");
    }
    return PET_OK;
}

pet_status pet_batch_create(pet_state *const *states, int32_t n, pet_batch **out) {
    if (!states || !out || n < 1) return set_error(PET_ERR_INVALID, "need at least one state");
    *out = nullptr;
    for (int j = 0; j < n; ++j) {
        if (!states[j]) return set_error(PET_ERR_INVALID, "null state in batch");
        if (states[j]->prob->plan->nz != 1 || states[j]->prob->plan->ring)
            return set_error(PET_ERR_INVALID, "batches take single-slice images");
        for (int i = 0; i < j; ++i)
            if (states[i] == states[j]) return set_error(PET_ERR_INVALID, "a state appears twice in the batch");
    }
    pet_batch *b = new (std::nothrow) pet_batch();
    if (!b) return set_error(PET_ERR_OOM, "host allocation failed");
    b->states.assign(states, states + n);
    b->members.resize(n);
    pet_status e;
    if ((e = dalloc(&b->d_members, (size_t)n, "batch members")) != PET_OK) {
        pet_batch_destroy(b);
        return e;
    }
    // the objective pass: one segment per member (its full-data forward blocks), longest items first
    std::vector<WorkSeg> obj;
    for (int j = 0; j < n; ++j) {
        const pet_plan *pl = b->states[j]->prob->plan;
        obj.push_back({j, WK_FWD_OBJECTIVE, 0, forward_blocks(pl->M, 1, full_group(pl)), full_group(pl), 0});
    }
    std::stable_sort(obj.begin(), obj.end(), [&](const WorkSeg &x, const WorkSeg &y) {
        const pet_plan *px = b->states[x.member]->prob->plan, *py = b->states[y.member]->prob->plan;
        return (std::max(px->nx, px->ny) + x.shape - 1) / x.shape > (std::max(py->nx, py->ny) + y.shape - 1) / y.shape;
    });
    for (WorkSeg &g : obj) {
        g.first = b->n_obj_items;
        b->n_obj_items += g.count;
    }
    b->n_obj_segs = n;
    if ((e = dalloc(&b->d_obj_segs, (size_t)n, "batch objective segments")) != PET_OK ||
        (e = dalloc(&b->d_obj_claim, 1, "batch objective claim")) != PET_OK ||
        (e = dalloc(&b->d_status, 1, "batch status")) != PET_OK ||
        (e = cuda_ok(cudaMemset(b->d_status, 0, sizeof(int)), "batch status reset")) != PET_OK) {
        pet_batch_destroy(b);
        return e;
    }
    const cudaError_t ce = cudaMemcpy(b->d_obj_segs, obj.data(), sizeof(WorkSeg) * obj.size(),
                                      cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        pet_batch_destroy(b);
        return cuda_ok(ce, "batch objective segment upload");
    }
    *out = b;
    return PET_OK;
}

}  // extern "C"

namespace {

void fill_member(BatchMember &m, const pet_state *st, float alpha, const int *seq) {
    const pet_problem *p = st->prob;
    const pet_plan *pl = p->plan;
    m.views = pl->d_views;
    m.uc = pl->d_uc;
    m.order = pl->d_order;
    m.sub_off = pl->d_sub_off;
    m.nx = pl->nx;
    m.ny = pl->ny;
    m.nb = pl->nb;
    m.ns = pl->ns;
    m.sens_t = pl->d_sens_t;
    m.sens = pl->d_sens;
    m.g = p->d_g;
    m.w = p->d_w;
    m.w_scalar = p->w_scalar;
    m.beta = p->pen.beta;
    m.pot = p->pen.potential;
    m.delta = p->pen.delta;
    m.status = p->d_status;
    m.algo = st->algo;
    m.table_dtype = st->table_dtype;
    m.img = st->img;
    m.alt = st->alt;
    m.ratio = st->ratio;
    m.ratio_full = st->ratio_full;
    m.s_hat = st->s_hat;
    m.f_anc = st->f_anc;
    m.s_anc = st->s_anc;
    m.B = st->B;
    m.d = st->precond == PET_PRECOND_ITERATE ? nullptr : st->d;
    m.table = st->table;
    m.qbar = st->qbar;
    m.qtil = st->qtil;
    m.alpha = alpha;
    m.seq = seq;
    m.alphas = nullptr;
    m.na = pl->na;
    m.n_ll = forward_blocks(pl->M, 1, full_group(pl));
    m.part = st->d_part;
}

// Work segments of the persistent phases of n_iter batched updates (into
// b->h_segs and b->phases).  Per update:
//   forward: every member's subset rays, plus the rays of every view of the
//     members whose anchor pass is due (anchor items first: they are the
//     longest, so the dynamic claim order leaves short items for the tail);
//   at an anchor update: a back phase with the anchor back projections and
//     the other members' updates, the anchor finishes, then a back phase with
//     the anchored members' updates; otherwise one back phase with every
//     member's update.
// Back phases are split by potential class (the quadratic epilogue and the
// edge-preserving one are different kernels), longest tiles first.
// PET_BATCH_STREAMS: the batch's own streams (up to 8), created on first use;
// fork makes them wait for `s`, join makes `s` wait for them.
constexpr int kBatchSideStreams = 8;

pet_status batch_fork(pet_batch *b, cudaStream_t s) {
    if (b->side.empty()) {
        const int k = std::max(1, std::min((int)b->states.size(), kBatchSideStreams));
        PET_TRY(cuda_ok(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming), "event"));
        for (int i = 0; i < k; ++i) {
            cudaStream_t sd = nullptr;
            cudaEvent_t e = nullptr;
            PET_TRY(cuda_ok(cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking), "batch stream"));
            b->side.push_back(sd);
            PET_TRY(cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event"));
            b->side_ev.push_back(e);
        }
    }
    PET_TRY(cuda_ok(cudaEventRecord(b->fork_ev, s), "event record"));
    for (cudaStream_t sd : b->side) PET_TRY(cuda_ok(cudaStreamWaitEvent(sd, b->fork_ev, 0), "stream wait"));
    return PET_OK;
}

pet_status batch_join(pet_batch *b, cudaStream_t s) {
    for (size_t i = 0; i < b->side.size(); ++i) {
        PET_TRY(cuda_ok(cudaEventRecord(b->side_ev[i], b->side[i]), "event record"));
        PET_TRY(cuda_ok(cudaStreamWaitEvent(s, b->side_ev[i], 0), "stream wait"));
    }
    return PET_OK;
}

void build_batch_phases(pet_batch *b, int n_iter, const std::vector<std::vector<uint8_t>> &anchors) {
    const int n = (int)b->states.size();
    b->h_segs.clear();
    b->phases.assign((size_t)n_iter, {});
    int claim = 0;
    auto tiles_of = [](const pet_plan *pl) { return ((pl->nx + 15) / 16) * ((pl->ny + 15) / 16); };
    auto major_of = [](const pet_plan *pl) { return std::max(pl->nx, pl->ny); };
    auto emit = [&](int i, int kind, std::vector<WorkSeg> &segs, int genpot) {
        if (segs.empty()) return;
        pet_batch::Phase ph{kind, (int)b->h_segs.size(), (int)segs.size(), 0, 256, genpot, claim++};
        for (WorkSeg &g : segs) {
            g.first = ph.n_items;
            ph.n_items += g.count;
            if (kind == 1)
                ph.threads = std::max(ph.threads, back_block_threads(g.shape,
                                                                     b->states[g.member]->prob->plan->max_sub_views));
            b->h_segs.push_back(g);
        }
        b->phases[(size_t)i].push_back(ph);
    };
    for (int i = 0; i < n_iter; ++i) {
        bool any = false;
        std::vector<WorkSeg> fa, fu;
        for (int j = 0; j < n; ++j) {
            const pet_plan *pl = b->states[j]->prob->plan;
            if (anchors[j][i]) {
                any = true;
                fa.push_back({j, WK_FWD_ANCHOR, 0, forward_blocks(pl->M, 1, full_group(pl)), full_group(pl), 0});
            }
            fu.push_back({j, WK_FWD_UPDATE, 0, forward_blocks(max_sub_rays(pl), 1, choose_group(pl)),
                          choose_group(pl), 0});
        }
        // bands per chunk decide an item's length
        auto longer_fwd = [&](const WorkSeg &x, const WorkSeg &y) {
            const int lx = (major_of(b->states[x.member]->prob->plan) + x.shape - 1) / x.shape;
            const int ly = (major_of(b->states[y.member]->prob->plan) + y.shape - 1) / y.shape;
            return lx > ly;
        };
        std::stable_sort(fa.begin(), fa.end(), longer_fwd);
        std::stable_sort(fu.begin(), fu.end(), longer_fwd);
        fa.insert(fa.end(), fu.begin(), fu.end());
        emit(i, 0, fa, 0);
        // views per subset decide a back item's length
        auto longer_back = [&](const WorkSeg &x, const WorkSeg &y) {
            return b->states[x.member]->prob->plan->max_sub_views > b->states[y.member]->prob->plan->max_sub_views;
        };
        for (int pass = any ? 0 : 1; pass < 2; ++pass) {
            for (int gp = 0; gp < 2; ++gp) {
                std::vector<WorkSeg> anc, upd;
                for (int j = 0; j < n; ++j) {
                    const pet_state *st = b->states[j];
                    const pet_plan *pl = st->prob->plan;
                    const int member_gp = st->prob->pen.potential != PET_POT_QUADRATIC ? 1 : 0;
                    if (pass == 0 && anchors[j][i] && gp == 0)
                        anc.push_back({j, WK_BACK_ANCHOR, 0, tiles_of(pl) * pl->ns, pl->back_run, tiles_of(pl)});
                    const bool update_here = any ? ((pass == 0) != (anchors[j][i] != 0)) : true;
                    if (update_here && member_gp == gp)
                        upd.push_back({j, WK_BACK_UPDATE, 0, tiles_of(pl), pl->back_run, tiles_of(pl)});
                }
                std::stable_sort(anc.begin(), anc.end(), longer_back);
                std::stable_sort(upd.begin(), upd.end(), longer_back);
                anc.insert(anc.end(), upd.begin(), upd.end());
                emit(i, 1, anc, gp);
            }
            if (pass == 0) b->phases[(size_t)i].push_back({2, 0, 0, 0, 0, 0, -1});   // the anchor finishes
        }
    }
    b->n_claims = claim;
}

// The dependency-driven epoch's work list (into b->h_df): every stage of every
// member, merged stage by stage across members (each member's k-th stage
// before any member's (k+1)-th), with each stage's needs (see dataflow.cu).
// Returns the block size and whether the members use an edge-preserving
// potential (all must share one potential class).
int build_batch_dataflow(pet_batch *b, int n_iter, const std::vector<std::vector<uint8_t>> &anchors, bool *genpot) {
    const int n = (int)b->states.size();
    struct Stage {
        DfSeg seg;
        int dep0, dep1;   // indices into the member's own stage list (-1: none)
    };
    std::vector<std::vector<Stage>> lists((size_t)n);
    int threads = 256;
    *genpot = b->states[0]->prob->pen.potential != PET_POT_QUADRATIC;
    for (int j = 0; j < n; ++j) {
        const pet_state *st = b->states[j];
        const pet_plan *pl = st->prob->plan;
        const int tiles = ((pl->nx + 15) / 16) * ((pl->ny + 15) / 16);
        threads = std::max(threads, back_block_threads(pl->back_run, pl->max_sub_views));
        bool ready = st->s_hat_ready;
        int prev_b = -1;
        auto add = [&](int kind, int count, int shape, int iter, int flag, int d0, int d1) {
            DfSeg g{j, kind, 0, count, shape, tiles, iter, flag, -1, 0, -1, 0};
            lists[(size_t)j].push_back({g, d0, d1});
            return (int)lists[(size_t)j].size() - 1;
        };
        for (int i = 0; i < n_iter; ++i) {
            int fin = -1;
            if (anchors[j][i]) {
                const int af = add(DF_FWD_ANCHOR, forward_blocks(pl->M, 1, full_group(pl)), full_group(pl), i, 0,
                                   prev_b, -1);
                const int ab = add(DF_BACK_ANCHOR, tiles * pl->ns, pl->back_run, i, 0, af, -1);
                fin = add(DF_FINISH, (int)((plane_of(pl) + 255) / 256), 0, i,
                          st->algo == PET_ALGO_SVREM && !ready ? 1 : 0, ab, -1);
                if (st->algo == PET_ALGO_SVREM) ready = true;
            }
            const int f = add(DF_FWD_UPDATE, forward_blocks(max_sub_rays(pl), 1, choose_group(pl)),
                              choose_group(pl), i, 0, prev_b, -1);
            prev_b = add(DF_BACK_UPDATE, tiles, pl->back_run, i, 0, f, fin);
        }
    }
    // merge stage by stage; map each member's stage indices to list positions
    std::vector<std::vector<int>> pos((size_t)n);
    for (int j = 0; j < n; ++j) pos[(size_t)j].assign(lists[(size_t)j].size(), -1);
    b->h_df.clear();
    size_t longest = 0;
    for (const auto &l : lists) longest = std::max(longest, l.size());
    int items = 0;
    for (size_t k = 0; k < longest; ++k)
        for (int j = 0; j < n; ++j) {
            if (k >= lists[(size_t)j].size()) continue;
            Stage &stg = lists[(size_t)j][k];
            stg.seg.first = items;
            items += stg.seg.count;
            if (stg.dep0 >= 0) {
                stg.seg.dep0 = pos[(size_t)j][(size_t)stg.dep0];
                stg.seg.need0 = lists[(size_t)j][(size_t)stg.dep0].seg.count;
            }
            if (stg.dep1 >= 0) {
                stg.seg.dep1 = pos[(size_t)j][(size_t)stg.dep1];
                stg.seg.need1 = lists[(size_t)j][(size_t)stg.dep1].seg.count;
            }
            pos[(size_t)j][k] = (int)b->h_df.size();
            b->h_df.push_back(stg.seg);
        }
    return threads;
}

// The dependency-driven epoch on stream s: the iterate copy (odd update
// counts), SEM statistics due, the counters' reset, then one launch.
pet_status enqueue_batch_dataflow(pet_batch *b, int32_t n_iter, int threads, bool genpot, cudaStream_t s) {
    const bool odd = (n_iter % 2) == 1;
    if (odd)
        for (pet_state *st : b->states) {
            const long long plane = plane_of(st->prob->plan);
            PET_TRY(cuda_ok(cudaMemcpyAsync(st->alt, st->img, (size_t)plane * 4, cudaMemcpyDeviceToDevice, s),
                            "cudaMemcpyAsync"));
        }
    for (pet_state *st : b->states)
        if (st->algo == PET_ALGO_SEM && !st->s_hat_ready) {
            PET_TRY(sem_init(st, odd ? st->alt : st->img, s));
            st->s_hat_ready = true;
        }
    const int n_segs = (int)b->h_df.size();
    const DfSeg &last = b->h_df.back();
    PET_TRY(launch_zero_ints(b->d_df_done, n_segs + 1, s));
    return launch_dataflow_epoch(b->d_members, b->d_df, n_segs, last.first + last.count, odd ? 1 : 0, b->d_df_done,
                                 b->d_status, b->wait_limit, genpot, threads, s);
}

// All launches of one batched epoch on stream s (phases from build_batch_phases).
pet_status enqueue_batch_epoch(pet_batch *b, int32_t n_iter, const std::vector<std::vector<uint8_t>> &anchors,
                               cudaStream_t s) {
    const int n = (int)b->states.size();
    const bool odd = (n_iter % 2) == 1;
    if (odd)
        for (pet_state *st : b->states) {
            const long long plane = plane_of(st->prob->plan);
            PET_TRY(cuda_ok(cudaMemcpyAsync(st->alt, st->img, (size_t)plane * 4, cudaMemcpyDeviceToDevice, s),
                            "cudaMemcpyAsync"));
        }
    PET_TRY(launch_zero_ints(b->d_claims, b->n_claims, s));
    for (int i = 0; i < n_iter; ++i) {
        const bool in_is_img = ((i % 2) == 0) != odd;
        for (int j = 0; j < n; ++j) {
            pet_state *st = b->states[j];
            if (st->algo == PET_ALGO_SEM && !st->s_hat_ready) {
                PET_TRY(sem_init(st, in_is_img ? st->img : st->alt, s));
                st->s_hat_ready = true;
            }
        }
        for (const pet_batch::Phase &ph : b->phases[(size_t)i]) {
            if (ph.kind == 0) {
                PET_TRY(launch_persistent_forward(b->d_members, b->d_segs + ph.seg_off, ph.n_segs, ph.n_items, i,
                                                  in_is_img ? 1 : 0, b->d_claims + ph.claim, false, s));
            } else if (ph.kind == 1) {
                PET_TRY(launch_persistent_back(b->d_members, b->d_segs + ph.seg_off, ph.n_segs, ph.n_items, i,
                                               in_is_img ? 1 : 0, b->d_claims + ph.claim, ph.genpot != 0, ph.threads,
                                               s));
            } else {
                for (int j = 0; j < n; ++j) {
                    if (!anchors[j][i]) continue;
                    pet_state *st = b->states[j];
                    const pet_plan *pl = st->prob->plan;
                    const long long plane = plane_of(pl);
                    const float *in = in_is_img ? st->img : st->alt;
                    if (st->algo == PET_ALGO_SVREM) {
                        PET_TRY(launch_svrem_anchor_finish(st->B, pl->ns, plane, pl->nz, in, st->f_anc, st->s_anc,
                                                           st->s_hat, !st->s_hat_ready, s));
                        st->s_hat_ready = true;
                    } else {
                        PET_TRY(launch_svrg_anchor_finish(st->B, pl->ns, plane, pl->nz, pl->d_sens, st->qtil, s));
                    }
                }
            }
        }
    }
    return PET_OK;
}

}  // namespace

extern "C" {

pet_status pet_batch_epoch(pet_batch *b, const int32_t *h_seqs, int32_t n_iter, const float *h_alpha,
                           const int32_t *h_eta, void *stream) {
    if (!b || !h_alpha || !h_eta) return set_error(PET_ERR_INVALID, "null argument");
    const int n = (int)b->states.size();
    cudaStream_t s = (cudaStream_t)stream;
    if (n_iter < 0) return set_error(PET_ERR_INVALID, "n_iter must be >= 0");
    for (int j = 0; j < n; ++j) {
        PET_TRY(check_seq(b->states[j]->prob->plan, h_seqs ? h_seqs + (size_t)j * n_iter : nullptr, n_iter));
        if (!std::isfinite(h_alpha[j])) return set_error(PET_ERR_INVALID, "alpha must be finite");
        const int algo = b->states[j]->algo;
        if ((algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG) && h_eta[j] < 1)
            return set_error(PET_ERR_INVALID, "eta must be >= 1");
    }
    if (n_iter == 0) return PET_OK;
    if (b->mode == PET_BATCH_STREAMS) {
        // every member's own epoch call (its captured graphs), member j on the batch's stream j mod k
        PET_TRY(batch_fork(b, s));
        for (int j = 0; j < n; ++j) {
            pet_state *st = b->states[j];
            const int algo = st->algo;
            PET_TRY(epoch_common(st, algo, h_seqs + (size_t)j * n_iter, n_iter,
                                 algo == PET_ALGO_OSEM ? 0.0f : h_alpha[j], 0.0f,
                                 (algo == PET_ALGO_SVREM || algo == PET_ALGO_SVRG) ? h_eta[j] : 1,
                                 b->side[(size_t)j % b->side.size()]));
        }
        return batch_join(b, s);
    }
    const size_t need = (size_t)n * n_iter;
    if ((int)need > b->seq_cap) {
        int *grown = nullptr;
        float *grown_a = nullptr;
        PET_TRY(dalloc(&grown, need, "batch subset sequences"));
        if (dalloc(&grown_a, need, "batch step sizes") != PET_OK) {
            dfree(grown);
            return PET_ERR_OOM;
        }
        if (b->d_seqs) {
            PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
            dfree(b->d_seqs);
            dfree(b->d_alphas);
        }
        b->d_seqs = grown;
        b->d_alphas = grown_a;
        b->seq_cap = (int)need;
    }
    std::vector<float> alphas(need);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n_iter; ++i) alphas[(size_t)j * n_iter + i] = h_alpha[j];
    PET_TRY(cuda_ok(cudaMemcpyAsync(b->d_seqs, h_seqs, sizeof(int32_t) * need, cudaMemcpyHostToDevice, s),
                    "batch sequence copy"));
    PET_TRY(cuda_ok(cudaMemcpyAsync(b->d_alphas, alphas.data(), sizeof(float) * need, cudaMemcpyHostToDevice, s),
                    "batch step size copy"));
    for (int j = 0; j < n; ++j) {
        fill_member(b->members[j], b->states[j], h_alpha[j], b->d_seqs + (size_t)j * n_iter);
        b->members[j].alphas = b->d_alphas + (size_t)j * n_iter;
    }
    PET_TRY(cuda_ok(cudaMemcpyAsync(b->d_members, b->members.data(), sizeof(BatchMember) * n, cudaMemcpyHostToDevice,
                                    s),
                    "batch member copy"));
    std::vector<std::vector<uint8_t>> anchors(n, std::vector<uint8_t>((size_t)n_iter, 0));
    bool direct = !use_graphs() || profiling_enabled() || !b->graphs_on;
    std::vector<int64_t> key = {n_iter};
    for (int j = 0; j < n; ++j) {
        pet_state *st = b->states[j];
        if ((st->algo == PET_ALGO_SVREM || st->algo == PET_ALGO_SEM) && !st->s_hat_ready) direct = true;
        if (st->algo != PET_ALGO_SVREM && st->algo != PET_ALGO_SVRG) continue;
        for (int i = 0; i < n_iter; ++i)
            if ((st->k + i) % ((long long)h_eta[j] * st->prob->plan->ns) == 0) {
                anchors[j][i] = 1;
                key.push_back((int64_t)j * (1LL << 32) + i);
            }
    }
    bool uniform_potential = true;
    for (int j = 1; j < n; ++j)
        uniform_potential &= (b->states[j]->prob->pen.potential != PET_POT_QUADRATIC) ==
                             (b->states[0]->prob->pen.potential != PET_POT_QUADRATIC);
    if (b->mode == PET_BATCH_DATAFLOW && uniform_potential) {
        bool genpot = false;
        const int threads = build_batch_dataflow(b, n_iter, anchors, &genpot);
        const int n_segs = (int)b->h_df.size();
        if (n_segs > b->df_cap || n_segs + 1 > b->df_done_cap) {
            DfSeg *grown = nullptr;
            int *grown_d = nullptr;
            PET_TRY(dalloc(&grown, (size_t)n_segs, "dataflow segments"));
            if (dalloc(&grown_d, (size_t)n_segs + 1, "dataflow counters") != PET_OK) {
                dfree(grown);
                return PET_ERR_OOM;
            }
            if (b->d_df) {
                PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
                dfree(b->d_df);
                dfree(b->d_df_done);
            }
            b->d_df = grown;
            b->d_df_done = grown_d;
            b->df_cap = n_segs;
            b->df_done_cap = n_segs + 1;
            for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
            b->graphs.clear();
        }
        PET_TRY(cuda_ok(cudaMemcpyAsync(b->d_df, b->h_df.data(), sizeof(DfSeg) * n_segs, cudaMemcpyHostToDevice, s),
                        "dataflow segment copy"));
        pet_status rc;
        key.push_back(-1);   // this mode's graphs apart from the phases'
        if (direct) {
            rc = enqueue_batch_dataflow(b, n_iter, threads, genpot, s);
        } else {
            pet_state holder{};
            holder.cap = b->cap;
            holder.graphs.swap(b->graphs);
            holder.graph_tick = b->graph_tick;
            rc = run_graph(&holder, key, s,
                           [&](cudaStream_t cs) { return enqueue_batch_dataflow(b, n_iter, threads, genpot, cs); });
            b->graphs.swap(holder.graphs);
            b->graph_tick = holder.graph_tick;
            b->cap = holder.cap;
            holder.cap = nullptr;
        }
        if (rc == PET_OK)
            for (int j = 0; j < n; ++j) {
                pet_state *st = b->states[j];
                if (st->algo == PET_ALGO_SVREM)
                    for (int i = 0; i < n_iter; ++i) st->s_hat_ready |= anchors[j][i] != 0;
                st->k += n_iter;
            }
        return rc;
    }
    build_batch_phases(b, n_iter, anchors);
    if ((int)b->h_segs.size() > b->seg_cap || b->n_claims > b->claim_cap) {
        WorkSeg *grown = nullptr;
        int *grown_c = nullptr;
        const size_t segs = std::max((size_t)b->seg_cap, b->h_segs.size());
        const size_t claims = (size_t)std::max(b->claim_cap, b->n_claims);
        PET_TRY(dalloc(&grown, segs, "batch work segments"));
        if (dalloc(&grown_c, claims, "batch claim counters") != PET_OK) {
            dfree(grown);
            return PET_ERR_OOM;
        }
        // the old buffers may still be read by enqueued work: release them after the stream drains
        if (b->d_segs) {
            PET_TRY(cuda_ok(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
            dfree(b->d_segs);
            dfree(b->d_claims);
        }
        b->d_segs = grown;
        b->d_claims = grown_c;
        b->seg_cap = (int)segs;
        b->claim_cap = (int)claims;
        // captured epochs hold the old pointers
        for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
        b->graphs.clear();
    }
    PET_TRY(cuda_ok(cudaMemcpyAsync(b->d_segs, b->h_segs.data(), sizeof(WorkSeg) * b->h_segs.size(),
                                    cudaMemcpyHostToDevice, s),
                    "batch work segment copy"));
    pet_status rc;
    if (direct) {
        rc = enqueue_batch_epoch(b, n_iter, anchors, s);
    } else {
        // a batch keeps its own graph cache; run_graph takes a state, so borrow
        // the cache of a stand-in state object
        pet_state holder{};
        holder.cap = b->cap;
        holder.graphs.swap(b->graphs);
        holder.graph_tick = b->graph_tick;
        rc = run_graph(&holder, key, s, [&](cudaStream_t cs) { return enqueue_batch_epoch(b, n_iter, anchors, cs); });
        b->graphs.swap(holder.graphs);
        b->graph_tick = holder.graph_tick;
        b->cap = holder.cap;
        holder.cap = nullptr;
    }
    if (rc == PET_OK)
        for (pet_state *st : b->states) st->k += n_iter;
    return rc;
}

pet_status pet_batch_objective_async(pet_batch *b, double *d_phi, void *stream) {
    if (!b || !d_phi) return set_error(PET_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)b->states.size();
    if (b->mode == PET_BATCH_STREAMS) {
        PET_TRY(batch_fork(b, s));
        for (int j = 0; j < n; ++j)
            PET_TRY(pet_state_objective_async(b->states[j], d_phi + 3 * j, b->side[(size_t)j % b->side.size()]));
        return batch_join(b, s);
    }
    // descriptors with the output slots (the subset sequences are not read here)
    int pen_blocks = 0;
    for (int j = 0; j < n; ++j) {
        fill_member(b->members[j], b->states[j], b->members[j].alpha, b->members[j].seq);
        b->members[j].phi = d_phi + 3 * j;
        const pet_plan *pl = b->states[j]->prob->plan;
        pen_blocks = std::max(pen_blocks, (pl->N + 255) / 256);
    }
    PET_TRY(cuda_ok(cudaMemcpyAsync(b->d_members, b->members.data(), sizeof(BatchMember) * n, cudaMemcpyHostToDevice,
                                    s),
                    "batch member copy"));
    PET_TRY(launch_zero_ints(b->d_obj_claim, 1, s));
    PET_TRY(launch_persistent_forward(b->d_members, b->d_obj_segs, b->n_obj_segs, b->n_obj_items, 0, 1,
                                      b->d_obj_claim, true, s));
    return launch_batch_objective_finish(b->d_members, n, pen_blocks, s);
}

pet_status pet_state_set_preconditioner(pet_state *st, int32_t kind) {
    if (!st) return set_error(PET_ERR_INVALID, "null state");
    if (st->algo != PET_ALGO_SAGA && st->algo != PET_ALGO_SVRG)
        return set_error(PET_ERR_INVALID, "the preconditioner choice applies to SAGA and SVRG states");
    if (kind != PET_PRECOND_CONSTANT && kind != PET_PRECOND_ITERATE)
        return set_error(PET_ERR_INVALID, "unknown preconditioner kind");
    if (kind != st->precond) {
        st->precond = kind;
        // captured epochs hold the old preconditioner pointer
        for (auto &g : st->graphs) cudaGraphExecDestroy(g.exec);
        st->graphs.clear();
    }
    return PET_OK;
}

pet_status pet_state_reset(pet_state *st, void *stream) {
    if (!st) return set_error(PET_ERR_INVALID, "null state");
    return state_init(st, (cudaStream_t)stream);
}

pet_status pet_state_sync(pet_state *st, void *stream) {
    if (!st) return set_error(PET_ERR_INVALID, "null state");
    return read_status(st->prob, (cudaStream_t)stream);
}

}  // extern "C"
