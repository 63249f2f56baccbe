// Back projection as a pixel-driven gather (K2), fused with the per-pixel
// update of each method (K3).
//
// b_n = sum_{m in S_t} a_mn r_m as a gather per pixel (no atomics, so the
// result is deterministic).  Single slices use tiles with runs of pixels
// that share each ray's band split (back_tile_kernel); slice stacks carry a
// block of 8 slices per thread; multi-ring volumes split each band piece over
// the layers its axial range crosses.  In each view only the bins whose ray
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
#include "petvr_internal.cuh"

namespace petvr {

namespace {

constexpr int kBlock = 256;
constexpr int kLanes = 4;           // slice stacks: lanes per (pixel, slice); each takes every 4th view
constexpr float kCandEps = 1e-3f;   // candidate-bin margin (pixels)
constexpr int kTile = 16;           // single slice: a block owns a kTile x kTile tile (kTile^2 == kBlock)
constexpr int kChunk = 16;          // views per shared-memory pass
constexpr int kTileBlockMax = 1024; // threads of a tile block: kTile * kTile / run per view of a chunk
static_assert(kTile * kTile == kBlock, "one pixel of the tile per thread");

struct Stencil {
    float cnt;   // sum_j d_nj, d_nj = gamma(f_n - f_j) (quadratic: the number of in-image neighbours)
    float sum;   // sum_j d_nj f_j
    float grad;  // dR/df_n = sum_j rho'(f_n - f_j)
};

// 4-neighbourhood of pixel (ix, iy) in slice z: surrogate weights and
// penalty gradient at f^k (out-of-image neighbours are dropped).  GENPOT
// selects the edge-preserving potentials (runtime pot); otherwise quadratic.
template <bool GENPOT>
__device__ __forceinline__ Stencil stencil4(const float *f, int ix, int iy, int nx, int ny, int nz, int z,
                                            float fk, int pot, float delta, int axial = 0) {
    const bool hl = ix > 0, hr = ix + 1 < nx, hd = iy > 0, hu = iy + 1 < ny;
    const bool hb = axial && z > 0, ht = axial && z + 1 < nz;        // axial neighbours of a volume
    const long long c = ((long long)iy * nx + ix) * nz + z;
    const float fl = hl ? __ldg(f + c - nz) : 0.0f;
    const float fr = hr ? __ldg(f + c + nz) : 0.0f;
    const float fd = hd ? __ldg(f + c - (long long)nx * nz) : 0.0f;
    const float fu = hu ? __ldg(f + c + (long long)nx * nz) : 0.0f;
    const float fb = hb ? __ldg(f + c - 1) : 0.0f;
    const float ft = ht ? __ldg(f + c + 1) : 0.0f;
    Stencil s{0.0f, 0.0f, 0.0f};
    if (!GENPOT) {
        // missing neighbours add exact zeros
        s.cnt = (float)((int)hl + (int)hr + (int)hd + (int)hu + (int)hb + (int)ht);
        s.sum = ((((fl + fr) + fd) + fu) + fb) + ft;
        s.grad = fk * s.cnt - s.sum;
        return s;
    }
    float dr, g;
    if (hl) { potential_dg(pot, delta, fk - fl, dr, g); s.cnt += g; s.sum += g * fl; s.grad += dr; }
    if (hr) { potential_dg(pot, delta, fk - fr, dr, g); s.cnt += g; s.sum += g * fr; s.grad += dr; }
    if (hd) { potential_dg(pot, delta, fk - fd, dr, g); s.cnt += g; s.sum += g * fd; s.grad += dr; }
    if (hu) { potential_dg(pot, delta, fk - fu, dr, g); s.cnt += g; s.sum += g * fu; s.grad += dr; }
    if (hb) { potential_dg(pot, delta, fk - fb, dr, g); s.cnt += g; s.sum += g * fb; s.grad += dr; }
    if (ht) { potential_dg(pot, delta, fk - ft, dr, g); s.cnt += g; s.sum += g * ft; s.grad += dr; }
    return s;
}

template <typename T> __device__ __forceinline__ float load_q(const void *p, long long i);
template <> __device__ __forceinline__ float load_q<float>(const void *p, long long i) {
    return static_cast<const float *>(p)[i];
}
template <> __device__ __forceinline__ float load_q<__nv_bfloat16>(const void *p, long long i) {
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
}
template <typename T> __device__ __forceinline__ float round_q(float x);
template <> __device__ __forceinline__ float round_q<float>(float x) { return x; }
template <> __device__ __forceinline__ float round_q<__nv_bfloat16>(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}
template <typename T> __device__ __forceinline__ void store_q(void *p, long long i, float x);
template <> __device__ __forceinline__ void store_q<float>(void *p, long long i, float x) {
    static_cast<float *>(p)[i] = x;
}
template <> __device__ __forceinline__ void store_q<__nv_bfloat16>(void *p, long long i, float x) {
    static_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(x);
}

// Per-pixel update after the gather: b = acc is A_t^T r_t at (pixel n, slice z).
template <int EPI, typename TQ, bool GENPOT>
__device__ __forceinline__ void apply_epilogue(const BackArgs &a, int t, long long i, int n, int ix, int iy,
                                               int z, float acc) {
    const long long plane = (long long)a.nx * a.ny * a.nz;
    // sensitivities: per pixel (shared by the slices of a stack) or per voxel
    const long long splane = a.axial ? plane : (long long)a.nx * a.ny;
    const long long sidx = a.axial ? i : (long long)n;
    const float inv_ns = 1.0f / (float)a.ns;
    const float alpha = a.alpha_dev ? __ldg(a.alpha_dev) : a.alpha;
    if (EPI == EPI_PLAIN) {
        a.out[i] = acc;
    } else if (EPI == EPI_ANCHOR) {
        a.out[(long long)t * plane + i] = acc;
    } else if (EPI == EPI_OSEM) {
        const float fk = a.f[i];
        const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float bp = a.beta * inv_ns;
        const float S = __ldg(a.sens_t + (long long)t * splane + sidx);
        const float c = bp * fmaf(fk, st.cnt, st.sum) - S;
        a.f_out[i] = m_step_root(fk * acc, S, bp * st.cnt, c);
    } else if (EPI == EPI_SVREM) {
        const float fk = a.f[i];
        const float ns = (float)a.ns;
        const float Bt = a.B[(long long)t * plane + i];
        const float tau = ns * fk * acc - ns * a.f_anc[i] * Bt + a.s_anc[i];
        const float s = fmaf(alpha, tau, (1.0f - alpha) * a.s_hat[i]);
        a.s_hat[i] = s;
        const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float S = __ldg(a.sens + sidx);
        const float c = a.beta * fmaf(fk, st.cnt, st.sum) - S;
        a.f_out[i] = m_step_root(s, S, a.beta * st.cnt, c);
    } else if (EPI == EPI_SAGA || EPI == EPI_SAGA_INIT) {
        const float fk = a.f[i];
        const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float gradR = st.grad;
        const float S = __ldg(a.sens_t + (long long)t * splane + sidx);
        const float q = round_q<TQ>(acc - S - a.beta * inv_ns * gradR);
        const long long qi = (long long)t * plane + i;
        if (EPI == EPI_SAGA_INIT) {
            store_q<TQ>(a.table, qi, q);
        } else {
            const float q_old = load_q<TQ>(a.table, qi);
            const float qb = a.qbar[i];
            const float dn = a.d ? a.d[i] : (S > 0.0f ? fk / S : 0.0f);    // d(f^(0)) or d_t(f^k)
            const float step = fmaf(alpha * dn, q - q_old + qb, fk);
            a.f_out[i] = fmaxf(step, 0.0f);
            a.qbar[i] = fmaf(q - q_old, inv_ns, qb);
            store_q<TQ>(a.table, qi, q);
        }
    } else if (EPI == EPI_SVRG) {
        const float fk = a.f[i];
        const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float gradR = st.grad;
        const float Bt = a.B[(long long)t * plane + i];
        const float dir = acc - Bt - a.beta * inv_ns * gradR + a.qtil[i];
        float dn;                                                   // d(f^(0)) or d_t(f^k)
        if (a.d) {
            dn = a.d[i];
        } else {
            const float S = __ldg(a.sens_t + (long long)t * splane + sidx);
            dn = S > 0.0f ? fk / S : 0.0f;
        }
        a.f_out[i] = fmaxf(fmaf(alpha * dn, dir, fk), 0.0f);
    } else if (EPI == EPI_SGA) {
        const float fk = a.f[i];
        const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float S = __ldg(a.sens_t + (long long)t * splane + sidx);
        const float dir = acc - S - a.beta * inv_ns * st.grad;      // grad Phi_t
        const float dt = S > 0.0f ? fk / S : 0.0f;                  // d_t(f) = f / A_t^T 1
        a.f_out[i] = fmaxf(fmaf(alpha * dt, dir, fk), 0.0f);
    } else if (EPI == EPI_SEM) {
        const float fk = a.f[i];
        const float s = fmaf(alpha, (float)a.ns * fk * acc, (1.0f - alpha) * a.s_hat[i]);
        a.s_hat[i] = s;
        const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float S = __ldg(a.sens + sidx);
        const float c = a.beta * fmaf(fk, st.cnt, st.sum) - S;
        a.f_out[i] = m_step_root(s, S, a.beta * st.cnt, c);
    } else if (EPI == EPI_SEM_INIT) {
        a.s_hat[i] = a.f[i] * acc;
    } else if (EPI == EPI_SAGAEM || EPI == EPI_SAGAEM_INIT) {
        const float fk = a.f[i];
        const float tau = (float)a.ns * fk * acc;                   // tau_t(f^k)
        float *T = static_cast<float *>(a.table);
        const long long ti = (long long)t * plane + i;
        if (EPI == EPI_SAGAEM_INIT) {
            T[ti] = tau;
        } else {
            const float T_old = T[ti];
            const float Tb = a.qbar[i];
            const float s = fmaf(alpha, tau - T_old + Tb, (1.0f - alpha) * a.s_hat[i]);
            a.s_hat[i] = s;
            const Stencil st = stencil4<GENPOT>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
            const float S = __ldg(a.sens + sidx);
            const float c = a.beta * fmaf(fk, st.cnt, st.sum) - S;
            a.f_out[i] = m_step_root(s, S, a.beta * st.cnt, c);
            a.qbar[i] = fmaf(tau - T_old, inv_ns, Tb);
            T[ti] = tau;
        }
    }
}

// Candidate bins of view vp whose band-kc interval can overlap the minor
// pixels [m_lo, m_hi): the bin positions uc0 + j K are approximate, so the
// range carries a margin far above their rounding.
__device__ __forceinline__ void candidate_bins(const ViewParams &vp, float kc, float m_lo, float m_hi, int nb,
                                               int &jlo, int &jhi) {
    const float base = fmaf(kc, vp.du, vp.uc0);
    const float e1 = (m_lo - fmaxf(vp.du, 0.0f) - base - kCandEps) * vp.invK;
    const float e2 = (m_hi - fminf(vp.du, 0.0f) - base + kCandEps) * vp.invK;
    jlo = max(0, (int)ceilf(fminf(e1, e2)));
    jhi = min(nb - 1, (int)floorf(fmaxf(e1, e2)));
}

// Stage the views [vb, vb + nv) of `order` into shared memory.
__device__ __forceinline__ void stage_views(const BackArgs &a, int vb, int nv, ViewParams *s_views, int *s_vid) {
    for (int q = threadIdx.x; q < nv; q += kBlock) {
        const int v = __ldg(a.order + vb + q);
        s_vid[q] = v;
        s_views[q] = a.views[v];
    }
}

// Slice-stack path: the geometry is shared by every slice, so a thread takes
// a block of kSliceBlock consecutive slices of one pixel (sums in registers)
// and kLanes lanes share the subset's views (lane l takes views l, l+4, ...).
// Each candidate bin's band piece is found once per slice block; the ratios
// of its slices are contiguous ([view][bin][z]).  After the lane sum, lane l
// applies the update to slices l, l + kLanes, ... of the block.
constexpr int kSliceBlock = 8;

template <int EPI, typename TQ, bool GENPOT>
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
    const int nzb = (a.nz + kSliceBlock - 1) / kSliceBlock;
    const int gid = blockIdx.x * kBlock + threadIdx.x;
    const int lane = gid % kLanes;
    const int rest = gid / kLanes;
    const int z0 = (rest % nzb) * kSliceBlock;
    const int n = rest / nzb;                            // pixel
    const bool live = n < a.nx * a.ny;
    const int ix = n % a.nx;
    const int iy = n / a.nx;
    const int zc = min(kSliceBlock, a.nz - z0);          // slices in this block

    float acc[kSliceBlock];
#pragma unroll
    for (int zz = 0; zz < kSliceBlock; ++zz) acc[zz] = 0.0f;
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
            const float *rv = a.r + (vb + q - r_view0) * a.nb * a.nz + z0;
            for (int j = jlo; j <= jhi; ++j) {
                const float2 u = __ldg(ucv + j);
                float fl, w0, w1;
                band_split(vp, band_point(vp, u.y, kc), band_point(vp, u.y, kc + 1.0f), fl, w0, w1);
                const int c0 = (int)fl + (int)u.x;
                const float w = (c0 == mrel) ? w0 : ((c0 + 1 == mrel) ? w1 : 0.0f);
                if (w == 0.0f) continue;
                const float *rj = rv + j * a.nz;
#pragma unroll
                for (int zz = 0; zz < kSliceBlock; ++zz)
                    if (zz < zc) acc[zz] = fmaf(w, __ldg(rj + zz), acc[zz]);
            }
        }
    }
#pragma unroll
    for (int zz = 0; zz < kSliceBlock; ++zz)
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) acc[zz] += __shfl_xor_sync(0xffffffffu, acc[zz], o);
    if (!live) return;
#pragma unroll
    for (int zz = 0; zz < kSliceBlock; ++zz)
        if (zz % kLanes == lane && zz < zc)
            apply_epilogue<EPI, TQ, GENPOT>(a, t, (long long)n * a.nz + z0 + zz, n, ix, iy, z0 + zz, acc[zz]);
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
// applies the update to layers l, l + kLanes, ...
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
#pragma unroll
    for (int iz = 0; iz < LMAX; ++iz)
        if (iz % kLanes == lane && iz < L) apply_epilogue<EPI, TQ, GENPOT>(a, t, n * L + iz, n, ix, iy, iz, acc[iz]);
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
template <int EPI, typename TQ, int kRun, bool GENPOT>
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
                const float r = __ldg(rv + j);
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
    if (threadIdx.x >= kTile * kTile) return;
    const int ix = x0 + (threadIdx.x % kTile);
    const int iy = y0 + (threadIdx.x / kTile);
    if (ix >= a.nx || iy >= a.ny) return;
    const int n = iy * a.nx + ix;
    apply_epilogue<EPI, TQ, GENPOT>(a, t, n, n, ix, iy, 0, acc);
}

template <int EPI, typename TQ, int kRun, bool GENPOT>
__global__ void __launch_bounds__(kTileBlockMax) back_tile_kernel(const BackArgs a) {
    const int t = a.t_dev ? __ldg(a.t_dev) : a.t0 + (int)blockIdx.y;
    back_tile_body<EPI, TQ, kRun, GENPOT>(a, t, blockIdx.x);
}

// Batched back projection + update: blockIdx.y picks the member, whose
// algorithm and table type select the epilogue; same body as the single
// launch, so each member's update is bit-identical to an unbatched one.
template <int kRun, bool GENPOT>
__global__ void __launch_bounds__(kTileBlockMax) batch_back_kernel(const BatchMember *ms, const int *idx, int iter,
                                                                   int in_is_img) {
    const BatchMember &m = ms[__ldg(idx + blockIdx.y)];
    const int tiles = ((m.nx + kTile - 1) / kTile) * ((m.ny + kTile - 1) / kTile);
    if ((int)blockIdx.x >= tiles) return;
    BackArgs b{};
    b.views = m.views;
    b.uc = m.uc;
    b.order = m.order;
    b.sub_off = m.sub_off;
    b.t_dev = m.seq + iter;
    b.nx = m.nx;
    b.ny = m.ny;
    b.nz = 1;
    b.nb = m.nb;
    b.ns = m.ns;
    b.run = kRun;
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
    const int t = __ldg(m.seq + iter);
    switch (m.algo) {
        case PET_ALGO_OSEM: back_tile_body<EPI_OSEM, float, kRun, GENPOT>(b, t, blockIdx.x); break;
        case PET_ALGO_SVREM: back_tile_body<EPI_SVREM, float, kRun, GENPOT>(b, t, blockIdx.x); break;
        case PET_ALGO_SAGA:
            if (m.table_dtype == PET_TABLE_BF16)
                back_tile_body<EPI_SAGA, __nv_bfloat16, kRun, GENPOT>(b, t, blockIdx.x);
            else
                back_tile_body<EPI_SAGA, float, kRun, GENPOT>(b, t, blockIdx.x);
            break;
        case PET_ALGO_SGA: back_tile_body<EPI_SGA, float, kRun, GENPOT>(b, t, blockIdx.x); break;
        case PET_ALGO_SEM: back_tile_body<EPI_SEM, float, kRun, GENPOT>(b, t, blockIdx.x); break;
        case PET_ALGO_SAGAEM: back_tile_body<EPI_SAGAEM, float, kRun, GENPOT>(b, t, blockIdx.x); break;
        default: back_tile_body<EPI_SVRG, float, kRun, GENPOT>(b, t, blockIdx.x); break;
    }
}

constexpr bool uses_stencil(int epi) {
    return epi == EPI_OSEM || epi == EPI_SVREM || epi == EPI_SAGA || epi == EPI_SAGA_INIT || epi == EPI_SVRG ||
           epi == EPI_SGA || epi == EPI_SEM || epi == EPI_SAGAEM;
}

template <int EPI, typename TQ, bool GENPOT>
pet_status go_impl(const BackArgs &a, int ny_grid, cudaStream_t s, int max_views) {
    if (a.axial && a.nz <= 8) {
        const int threads = a.nx * a.ny * kLanes;
        const dim3 grid((unsigned)((threads + kBlock - 1) / kBlock), (unsigned)ny_grid);
        const size_t smem = (size_t)max_views * (sizeof(ViewParams) + sizeof(int));
        if (a.nz <= 4)
            ring_back_column_kernel<EPI, TQ, GENPOT, 4><<<grid, kBlock, smem, s>>>(a);
        else
            ring_back_column_kernel<EPI, TQ, GENPOT, 8><<<grid, kBlock, smem, s>>>(a);
        return check_launch("ring_back_column_kernel");
    }
    if (a.axial) {
        const long long threads = (long long)a.nx * a.ny * a.nz * kLanes;
        const dim3 grid((unsigned)((threads + kBlock - 1) / kBlock), (unsigned)ny_grid);
        const size_t smem = (size_t)max_views * (sizeof(ViewParams) + sizeof(int));
        ring_back_kernel<EPI, TQ, GENPOT><<<grid, kBlock, smem, s>>>(a);
        return check_launch("ring_back_kernel");
    }
    if (a.nz == 1) {
        const int tiles = ((a.nx + kTile - 1) / kTile) * ((a.ny + kTile - 1) / kTile);
        const dim3 grid((unsigned)tiles, (unsigned)ny_grid);
        const size_t smem = (size_t)kChunk * (kTile * kTile * sizeof(float) + sizeof(ViewParams) + sizeof(int));
        // one thread per run: kTile * kTile / run runs per view of the largest chunk
        const int run = a.run == 4 ? 4 : 8;
        const int per_view = kTile * (kTile / run);
        const int threads = max(kTile * kTile, per_view * min(max_views, kChunk));
        launch_dependent(run == 4 ? back_tile_kernel<EPI, TQ, 4, GENPOT> : back_tile_kernel<EPI, TQ, 8, GENPOT>,
                         grid, dim3((unsigned)threads), smem, s, a);
        return check_launch("back_tile_kernel");
    }
    const long long threads = (long long)a.nx * a.ny * ((a.nz + kSliceBlock - 1) / kSliceBlock) * kLanes;
    const dim3 grid((unsigned)((threads + kBlock - 1) / kBlock), (unsigned)ny_grid);
    const size_t smem = (size_t)max_views * (sizeof(ViewParams) + sizeof(int));
    back_stack_kernel<EPI, TQ, GENPOT><<<grid, kBlock, smem, s>>>(a);
    return check_launch("back_stack_kernel");
}

template <int EPI, typename TQ>
pet_status go(const BackArgs &a, int ny_grid, cudaStream_t s, int max_views) {
    if constexpr (uses_stencil(EPI)) {
        if (a.pot != PET_POT_QUADRATIC) return go_impl<EPI, TQ, true>(a, ny_grid, s, max_views);
    }
    return go_impl<EPI, TQ, false>(a, ny_grid, s, max_views);
}

}  // namespace

pet_status launch_batch_back(const BatchMember *d_members, const int *d_idx, int n_members, int run, int tiles,
                             int max_views, int iter, int in_is_img, bool general_potential, cudaStream_t s) {
    if (n_members == 0 || tiles == 0) return PET_OK;
    const size_t smem = (size_t)kChunk * (kTile * kTile * sizeof(float) + sizeof(ViewParams) + sizeof(int));
    const int per_view = kTile * (kTile / run);
    const int threads = max(kTile * kTile, per_view * min(max_views, kChunk));
    const dim3 grid((unsigned)tiles, (unsigned)n_members);
    void (*k)(const BatchMember *, const int *, int, int) =
        general_potential ? (run == 4 ? batch_back_kernel<4, true> : batch_back_kernel<8, true>)
                          : (run == 4 ? batch_back_kernel<4, false> : batch_back_kernel<8, false>);
    launch_dependent(k, grid, dim3((unsigned)threads), smem, s, d_members, d_idx, iter, in_is_img);
    return check_launch("batch_back_kernel");
}

pet_status launch_back(const BackArgs &a, int epi, int table_dtype, int n_subsets_grid,
                       cudaStream_t s, int max_views) {
    const bool bf = table_dtype == PET_TABLE_BF16;
    const int g = n_subsets_grid;
    const int mv = max_views;
    ProfileScope prof(g > 1 ? 2 : 1, s);
    switch (epi) {
        case EPI_PLAIN: return go<EPI_PLAIN, float>(a, g, s, mv);
        case EPI_OSEM: return go<EPI_OSEM, float>(a, g, s, mv);
        case EPI_SVREM: return go<EPI_SVREM, float>(a, g, s, mv);
        case EPI_SVRG: return go<EPI_SVRG, float>(a, g, s, mv);
        case EPI_ANCHOR: return go<EPI_ANCHOR, float>(a, g, s, mv);
        case EPI_SAGA: return bf ? go<EPI_SAGA, __nv_bfloat16>(a, g, s, mv) : go<EPI_SAGA, float>(a, g, s, mv);
        case EPI_SAGA_INIT:
            return bf ? go<EPI_SAGA_INIT, __nv_bfloat16>(a, g, s, mv) : go<EPI_SAGA_INIT, float>(a, g, s, mv);
        case EPI_SGA: return go<EPI_SGA, float>(a, g, s, mv);
        case EPI_SEM: return go<EPI_SEM, float>(a, g, s, mv);
        case EPI_SEM_INIT: return go<EPI_SEM_INIT, float>(a, g, s, mv);
        case EPI_SAGAEM: return go<EPI_SAGAEM, float>(a, g, s, mv);
        case EPI_SAGAEM_INIT: return go<EPI_SAGAEM_INIT, float>(a, g, s, mv);
        default: return set_error(PET_ERR_INVALID, "back: unknown epilogue");
    }
}

}  // namespace petvr
