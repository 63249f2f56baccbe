// Small streaming kernels: data permutation, sensitivity sum, warm-start
// image, FP64 objective reduction, anchor and table bookkeeping.
#include "petvr_internal.cuh"

namespace petvr {

namespace {

constexpr int kBlock = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// dst[p][j][z] = src[order[p]][j][z]: natural view order -> subset-major order.
__global__ void permute_kernel(const float *src, float *dst, const int *order, int na, int nb, int nz) {
    const long long row = (long long)nb * nz;
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i >= row * na) return;
    const int p = (int)(i / row);
    const long long r = i % row;
    dst[i] = src[(long long)order[p] * row + r];
}

// sens = sum_t sens_t, summed in FP64.
__global__ void sum_sens_kernel(const float *sens_t, float *sens, int ns, int N) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= N) return;
    double s = 0.0;
    for (int t = 0; t < ns; ++t) s += sens_t[(long long)t * N + n];
    sens[n] = (float)s;
}

// Block-wide FP64 sum (kBlock threads); result valid in thread 0.
__device__ double block_sum(double v) {
    __shared__ double red[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kBlock / 32; ++i) s += red[i];
    __syncthreads();
    return s;
}

// out[z] = sum_m max(g_m - w_m, 0) for slice z (one block per slice), and
// out[nz] = sum_n sens_n (block nz).
__global__ void uniform_sums_kernel(const float *g, const float *w, float w_scalar, long long M, int nz,
                                    const float *sens, int N, double *out) {
    const int z = blockIdx.x;
    double s = 0.0;
    if (z < nz) {
        for (long long m = threadIdx.x; m < M; m += kBlock) {
            const long long idx = m * nz + z;
            const float d = g[idx] - (w ? w[idx] : w_scalar);
            s += d > 0.0f ? (double)d : 0.0;
        }
    } else {
        for (int n = threadIdx.x; n < N; n += kBlock) s += sens[n];
    }
    s = block_sum(s);
    if (threadIdx.x == 0) out[z] = s;
}

__global__ void uniform_fill_kernel(float *img, long long plane, int nz, const double *sums) {
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i >= plane) return;
    const double den = sums[nz];
    img[i] = den > 0.0 ? (float)(sums[i % nz] / den) : 0.0f;
}

// Per-block partial of R(f) = 1/2 sum_n sum_{j in N(n)} rho(f_n - f_j): each
// pixel adds half its potential terms (rho in FP32, sums in FP64).  N(n) is
// the in-plane 4-neighbourhood, plus the two axial neighbours when `axial`
// (a multi-ring volume; the slices of a stack are not coupled).
__global__ void penalty_partial_kernel(const float *f, int nx, int ny, int nz, int axial, int pot, float delta,
                                       double *part) {
    const long long plane = (long long)nx * ny * nz;
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    double r = 0.0;
    if (i < plane) {
        const int n = (int)(i / nz);
        const int z = (int)(i % nz);
        const int ix = n % nx, iy = n / nx;
        const bool hb = axial && z > 0, ht = axial && z + 1 < nz;
        const float fn = f[i];
        if (pot == PET_POT_QUADRATIC) {
            const double fd = fn;
            double acc = 0.0;
            if (ix > 0) { const double d = fd - f[i - nz]; acc += d * d; }
            if (ix + 1 < nx) { const double d = fd - f[i + nz]; acc += d * d; }
            if (iy > 0) { const double d = fd - f[i - (long long)nx * nz]; acc += d * d; }
            if (iy + 1 < ny) { const double d = fd - f[i + (long long)nx * nz]; acc += d * d; }
            if (hb) { const double d = fd - f[i - 1]; acc += d * d; }
            if (ht) { const double d = fd - f[i + 1]; acc += d * d; }
            r = 0.25 * acc;
        } else {
            double acc = 0.0;
            if (ix > 0) acc += potential_rho(pot, delta, fn - f[i - nz]);
            if (ix + 1 < nx) acc += potential_rho(pot, delta, fn - f[i + nz]);
            if (iy > 0) acc += potential_rho(pot, delta, fn - f[i - (long long)nx * nz]);
            if (iy + 1 < ny) acc += potential_rho(pot, delta, fn - f[i + (long long)nx * nz]);
            if (hb) acc += potential_rho(pot, delta, fn - f[i - 1]);
            if (ht) acc += potential_rho(pot, delta, fn - f[i + 1]);
            r = 0.5 * acc;
        }
    }
    r = block_sum(r);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// phi = sum(ll partials) - beta * sum(penalty partials), in one block, fixed order.
__global__ void objective_final_kernel(const double *ll, int n_ll, const double *pen, int n_pen, double beta,
                                       double *out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n_ll; i += kBlock) a += ll[i];
    for (int i = threadIdx.x; i < n_pen; i += kBlock) b += pen[i];
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        out[0] = a - beta * b;
        out[1] = a;
        out[2] = b;
    }
}

// SVREM anchor statistic s_anc = f_anc . sum_t B_t (the sum in FP64), with
// the anchor image f_anc taken from the current iterate f here (the anchor
// pass before this kernel reads f itself).
__global__ void svrem_finish_kernel(const float *B, int ns, long long plane, const float *f, float *f_anc,
                                    float *s_anc, float *s_hat, int init) {
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i >= plane) return;
    double s = 0.0;
    for (int t = 0; t < ns; ++t) s += B[(long long)t * plane + i];
    const float fa = f[i];
    f_anc[i] = fa;
    const float sa = (float)((double)fa * s);
    s_anc[i] = sa;
    if (init) s_hat[i] = sa;
}

__global__ void svrg_finish_kernel(const float *B, int ns, long long plane, int nz, const float *sens,
                                   float *qtil) {
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i >= plane) return;
    double s = 0.0;
    for (int t = 0; t < ns; ++t) s += B[(long long)t * plane + i];
    qtil[i] = (float)((s - (double)sens[i / nz]) / (double)ns);
}

template <typename TQ>
__device__ __forceinline__ double table_at(const void *tab, long long i);
template <> __device__ __forceinline__ double table_at<float>(const void *tab, long long i) {
    return static_cast<const float *>(tab)[i];
}
template <> __device__ __forceinline__ double table_at<__nv_bfloat16>(const void *tab, long long i) {
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(tab)[i]);
}

template <typename TQ>
__global__ void saga_finish_kernel(const void *tab, int ns, long long plane, float *qbar) {
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i >= plane) return;
    double s = 0.0;
    for (int t = 0; t < ns; ++t) s += table_at<TQ>(tab, (long long)t * plane + i);
    qbar[i] = (float)(s / (double)ns);
}

// d = N_s f0 / sens (0 where sens = 0): the constant preconditioner of §4.
__global__ void precond_kernel(const float *f0, const float *sens, int ns, long long plane, int nz, float *d) {
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i >= plane) return;
    const float s = sens[i / nz];
    d[i] = s > 0.0f ? (float)ns * f0[i] / s : 0.0f;
}

// Batched penalty partials (blockIdx.y = member) after the member's
// log-likelihood partials, then one block per member for the final sums.
__global__ void batch_penalty_kernel(const BatchMember *ms) {
    const BatchMember &m = ms[blockIdx.y];
    const int plane = m.nx * m.ny;
    if ((int)blockIdx.x * kBlock >= plane) return;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    double r = 0.0;
    if (i < plane) {
        const float *f = m.img;
        const int ix = i % m.nx, iy = i / m.nx;
        const float fn = f[i];
        if (m.pot == PET_POT_QUADRATIC) {
            const double fd = fn;
            double acc = 0.0;
            if (ix > 0) { const double d = fd - f[i - 1]; acc += d * d; }
            if (ix + 1 < m.nx) { const double d = fd - f[i + 1]; acc += d * d; }
            if (iy > 0) { const double d = fd - f[i - m.nx]; acc += d * d; }
            if (iy + 1 < m.ny) { const double d = fd - f[i + m.nx]; acc += d * d; }
            r = 0.25 * acc;
        } else {
            double acc = 0.0;
            if (ix > 0) acc += potential_rho(m.pot, m.delta, fn - f[i - 1]);
            if (ix + 1 < m.nx) acc += potential_rho(m.pot, m.delta, fn - f[i + 1]);
            if (iy > 0) acc += potential_rho(m.pot, m.delta, fn - f[i - m.nx]);
            if (iy + 1 < m.ny) acc += potential_rho(m.pot, m.delta, fn - f[i + m.nx]);
            r = 0.5 * acc;
        }
    }
    r = block_sum(r);
    if (threadIdx.x == 0) m.part[m.n_ll + blockIdx.x] = r;
}

__global__ void batch_objective_final_kernel(const BatchMember *ms) {
    const BatchMember &m = ms[blockIdx.x];
    const int n_pen = (m.nx * m.ny + kBlock - 1) / kBlock;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < m.n_ll; i += kBlock) a += m.part[i];
    for (int i = threadIdx.x; i < n_pen; i += kBlock) b += m.part[m.n_ll + i];
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        m.phi[0] = a - (double)m.beta * b;
        m.phi[1] = a;
        m.phi[2] = b;
    }
}

}  // namespace

// ---- launch shapes of the forward projectors (host) --------------------------

// Blocks of a forward launch over n_rays rays: single slices (nz == 1) run
// `group` band-chunk lanes per ray, slice stacks one warp (`group` chunks x 8
// z-lanes) per ray and slice window.  (Multi-ring launches pass nz = 1: a
// thread carries all ring pairs of its ray.)
int forward_blocks(int n_rays, int nz, int group) {
    const long long per_ray = nz > 1 ? (long long)stack_windows(nz) * 8 * group : group;
    const long long threads = (long long)n_rays * per_ray;
    return (int)((threads + kBlock - 1) / kBlock);
}

// Band chunks per ray for single slices and multi-ring lines: chunks of about
// 8 bands, as many as the image needs (slice stacks always use kStackChunks).
int default_chunks(int nx, int ny) {
    const int n = nx > ny ? nx : ny;
    if (n >= 160) return 32;
    if (n >= 80) return 16;
    return 8;
}

int choose_group(const pet_plan *plan) {
    if (plan->ring)                                                  // band chunks per line
        return plan->fwd_chunks > 0 ? plan->fwd_chunks : default_chunks(plan->nx, plan->ny);
    if (plan->nz > 1) return kStackChunks;                         // band chunks per ray and window
    return plan->fwd_chunks > 0 ? plan->fwd_chunks : default_chunks(plan->nx, plan->ny);
}

// Band chunks per ray of a full-data forward pass (anchor ratios, objectives,
// all-view projections) of a single-slice plan.  Such a grid is large, so the
// kernel is bound by instruction issue rather than latency, and each thread's
// fixed work (ray set-up, chunk reduction, epilogue) is better spread over
// more bands: the chunk count is halved from the plan's, down to 16, while the
// grid keeps at least kLargeGrid blocks and a chunk keeps at most kFullBands
// bands (8 chunks measured slower again on a 256^2 image: too few warps left
// to hide the load latency; on 512^2 images, 32 bands per chunk made the full
// pass 547 us against 426 us at the plan's 32 chunks, while 384^2 images, 24
// bands per chunk at 16 chunks, took 155 us against 168 us at 32).  Stacks
// and multi-ring plans keep theirs.
constexpr int kLargeGrid = 8 * 152;
constexpr int kFullBands = 24;

int full_group(const pet_plan *plan) {
    int g = choose_group(plan);
    if (plan->nz != 1 || plan->ring) return g;
    const int major = std::max(plan->nx, plan->ny);
    while (g > 16 && forward_blocks(plan->M, 1, g / 2) >= kLargeGrid && (major + g / 2 - 1) / (g / 2) <= kFullBands)
        g /= 2;
    return g;
}

pet_status launch_batch_objective_finish(const BatchMember *d_members, int n_members, int pen_blocks,
                                         cudaStream_t s) {
    if (n_members == 0) return PET_OK;
    batch_penalty_kernel<<<dim3((unsigned)pen_blocks, (unsigned)n_members), kBlock, 0, s>>>(d_members);
    pet_status st = check_launch("batch_penalty_kernel");
    if (st != PET_OK) return st;
    batch_objective_final_kernel<<<n_members, kBlock, 0, s>>>(d_members);
    return check_launch("batch_objective_final_kernel");
}

pet_status launch_permute_sino(const float *src, float *dst, const int *order, int na, int nb, int nz,
                               cudaStream_t s) {
    const long long n = (long long)na * nb * nz;
    if (n == 0) return PET_OK;
    permute_kernel<<<blocks_for(n), kBlock, 0, s>>>(src, dst, order, na, nb, nz);
    return check_launch("permute_kernel");
}

pet_status launch_sum_sens(const float *sens_t, float *sens, int ns, int N, cudaStream_t s) {
    sum_sens_kernel<<<blocks_for(N), kBlock, 0, s>>>(sens_t, sens, ns, N);
    return check_launch("sum_sens_kernel");
}

pet_status launch_uniform_image(const pet_problem *p, float *img, cudaStream_t s, double *sums) {
    const pet_plan *pl = p->plan;
    if (!sums) sums = p->d_scalar + 4;
    uniform_sums_kernel<<<pl->nz + 1, kBlock, 0, s>>>(p->d_g, p->d_w, p->w_scalar, (long long)pl->M, pl->nz,
                                                     pl->d_sens, pl->N, sums);
    pet_status st = check_launch("uniform_sums_kernel");
    if (st != PET_OK) return st;
    const long long plane = (long long)pl->N * pl->nz;
    uniform_fill_kernel<<<blocks_for(plane), kBlock, 0, s>>>(img, plane, pl->nz, sums);
    return check_launch("uniform_fill_kernel");
}

pet_status launch_objective_finish(const pet_problem *p, const float *img, int n_ll_blocks, double *part,
                                   double *d_out, cudaStream_t s) {
    const pet_plan *pl = p->plan;
    const long long plane = (long long)pl->N * pl->nz;
    const int n_pen = (int)blocks_for(plane);
    double *pen_part = part + n_ll_blocks;
    const int inner = pl->ring ? pl->layers : pl->nz;       // image entries per pixel
    penalty_partial_kernel<<<n_pen, kBlock, 0, s>>>(img, pl->nx, pl->ny, inner, pl->ring, p->pen.potential,
                                                    p->pen.delta, pen_part);
    pet_status st = check_launch("penalty_partial_kernel");
    if (st != PET_OK) return st;
    objective_final_kernel<<<1, kBlock, 0, s>>>(part, n_ll_blocks, pen_part, n_pen, (double)p->pen.beta,
                                                d_out);
    return check_launch("objective_final_kernel");
}

pet_status launch_objective_finish_raw(int nx, int ny, int nz, float beta, const float *img, int n_ll_blocks,
                                       double *part, double *d_out, cudaStream_t s) {
    const long long plane = (long long)nx * ny * nz;
    const int n_pen = (int)blocks_for(plane);
    double *pen_part = part + n_ll_blocks;
    penalty_partial_kernel<<<n_pen, kBlock, 0, s>>>(img, nx, ny, nz, 0, PET_POT_QUADRATIC, 1.0f, pen_part);
    pet_status st = check_launch("penalty_partial_kernel");
    if (st != PET_OK) return st;
    objective_final_kernel<<<1, kBlock, 0, s>>>(part, n_ll_blocks, pen_part, n_pen, (double)beta, d_out);
    return check_launch("objective_final_kernel");
}

pet_status launch_svrem_anchor_finish(const float *B, int ns, long long plane, int nz, const float *f,
                                      float *f_anc, float *s_anc, float *s_hat, bool init, cudaStream_t s) {
    (void)nz;
    svrem_finish_kernel<<<blocks_for(plane), kBlock, 0, s>>>(B, ns, plane, f, f_anc, s_anc, s_hat, init ? 1 : 0);
    return check_launch("svrem_finish_kernel");
}

pet_status launch_svrg_anchor_finish(const float *B, int ns, long long plane, int nz, const float *sens,
                                     float *qtil, cudaStream_t s) {
    svrg_finish_kernel<<<blocks_for(plane), kBlock, 0, s>>>(B, ns, plane, nz, sens, qtil);
    return check_launch("svrg_finish_kernel");
}

pet_status launch_saga_finish(const void *table, int table_dtype, int ns, long long plane, int nz,
                              const float *f0, const float *sens, float *qbar, float *d, cudaStream_t s) {
    if (table_dtype == PET_TABLE_BF16)
        saga_finish_kernel<__nv_bfloat16><<<blocks_for(plane), kBlock, 0, s>>>(table, ns, plane, qbar);
    else
        saga_finish_kernel<float><<<blocks_for(plane), kBlock, 0, s>>>(table, ns, plane, qbar);
    pet_status st = check_launch("saga_finish_kernel");
    if (st != PET_OK) return st;
    return launch_precond(f0, sens, ns, plane, nz, d, s);
}

pet_status launch_table_mean(const void *table, int table_dtype, int ns, long long plane, float *mean,
                             cudaStream_t s) {
    if (table_dtype == PET_TABLE_BF16)
        saga_finish_kernel<__nv_bfloat16><<<blocks_for(plane), kBlock, 0, s>>>(table, ns, plane, mean);
    else
        saga_finish_kernel<float><<<blocks_for(plane), kBlock, 0, s>>>(table, ns, plane, mean);
    return check_launch("table_mean_kernel");
}

pet_status launch_precond(const float *f0, const float *sens, int ns, long long plane, int nz, float *d,
                          cudaStream_t s) {
    precond_kernel<<<blocks_for(plane), kBlock, 0, s>>>(f0, sens, ns, plane, nz, d);
    return check_launch("precond_kernel");
}

}  // namespace petvr
