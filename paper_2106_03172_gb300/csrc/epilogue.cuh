// Device helpers shared by the back-projection kernels (backward.cu: single
// slices; volume.cu: slice stacks and multi-ring volumes): the penalty
// stencil, the per-pixel update of each method (the epilogue), candidate bins
// and view staging, and the dispatch from a runtime epilogue / table type /
// potential to the kernel template that handles it.
#pragma once

#include "petvr_internal.cuh"

namespace petvr {

namespace {

constexpr int kBlock = 256;
constexpr int kLanes = 4;           // multi-ring volumes: lanes per pixel column or voxel
constexpr float kCandEps = 1e-3f;   // candidate-bin margin (pixels)

// A float that may have been written earlier in the same kernel launch by
// another block (COH: a plain load, ordered by the reader's acquire) or that is
// read-only for the launch (the read-only data path).
template <bool COH>
__device__ __forceinline__ float ld_data(const float *p) {
    if (COH) return *p;
    return __ldg(p);
}

struct Stencil {
    float cnt;   // sum_j d_nj, d_nj = gamma(f_n - f_j) (quadratic: the number of in-image neighbours)
    float sum;   // sum_j d_nj f_j
    float grad;  // dR/df_n = sum_j rho'(f_n - f_j)
};

// Neighbourhood of pixel (ix, iy) in slice z (4 in the plane, plus the two
// axial neighbours of a volume when `axial`): surrogate weights and penalty
// gradient at f^k (out-of-image neighbours are dropped).  GENPOT selects the
// edge-preserving potentials (runtime pot); otherwise quadratic.
template <bool GENPOT, bool COH = false>
__device__ __forceinline__ Stencil stencil4(const float *f, int ix, int iy, int nx, int ny, int nz, int z,
                                            float fk, int pot, float delta, int axial = 0) {
    const bool hl = ix > 0, hr = ix + 1 < nx, hd = iy > 0, hu = iy + 1 < ny;
    const bool hb = axial && z > 0, ht = axial && z + 1 < nz;        // axial neighbours of a volume
    const long long c = ((long long)iy * nx + ix) * nz + z;
    const float fl = hl ? ld_data<COH>(f + c - nz) : 0.0f;
    const float fr = hr ? ld_data<COH>(f + c + nz) : 0.0f;
    const float fd = hd ? ld_data<COH>(f + c - (long long)nx * nz) : 0.0f;
    const float fu = hu ? ld_data<COH>(f + c + (long long)nx * nz) : 0.0f;
    const float fb = hb ? ld_data<COH>(f + c - 1) : 0.0f;
    const float ft = ht ? ld_data<COH>(f + c + 1) : 0.0f;
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
template <int EPI, typename TQ, bool GENPOT, bool COH = false>
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
        const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
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
        const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float S = __ldg(a.sens + sidx);
        const float c = a.beta * fmaf(fk, st.cnt, st.sum) - S;
        a.f_out[i] = m_step_root(s, S, a.beta * st.cnt, c);
    } else if (EPI == EPI_SAGA || EPI == EPI_SAGA_INIT) {
        const float fk = a.f[i];
        const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
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
        const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
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
        const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
        const float S = __ldg(a.sens_t + (long long)t * splane + sidx);
        const float dir = acc - S - a.beta * inv_ns * st.grad;      // grad Phi_t
        const float dt = S > 0.0f ? fk / S : 0.0f;                  // d_t(f) = f / A_t^T 1
        a.f_out[i] = fmaxf(fmaf(alpha * dt, dir, fk), 0.0f);
    } else if (EPI == EPI_SEM) {
        const float fk = a.f[i];
        const float s = fmaf(alpha, (float)a.ns * fk * acc, (1.0f - alpha) * a.s_hat[i]);
        a.s_hat[i] = s;
        const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
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
            const Stencil st = stencil4<GENPOT, COH>(a.f, ix, iy, a.nx, a.ny, a.nz, z, fk, a.pot, a.delta, a.axial);
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

constexpr bool uses_stencil(int epi) {
    return epi == EPI_OSEM || epi == EPI_SVREM || epi == EPI_SAGA || epi == EPI_SAGA_INIT || epi == EPI_SVRG ||
           epi == EPI_SGA || epi == EPI_SEM || epi == EPI_SAGAEM;
}

// Calls launcher.template run<EPI, TQ, GENPOT>() for a runtime epilogue,
// table type and potential (the general-potential forms only where the
// epilogue reads the penalty stencil).
template <int EPI, typename TQ, class Launcher>
pet_status with_potential(int pot, const Launcher &l) {
    if constexpr (uses_stencil(EPI)) {
        if (pot != PET_POT_QUADRATIC) return l.template run<EPI, TQ, true>();
    }
    return l.template run<EPI, TQ, false>();
}

template <class Launcher>
pet_status with_epilogue(int epi, int table_dtype, int pot, const Launcher &l) {
    const bool bf = table_dtype == PET_TABLE_BF16;
    switch (epi) {
        case EPI_PLAIN: return with_potential<EPI_PLAIN, float>(pot, l);
        case EPI_OSEM: return with_potential<EPI_OSEM, float>(pot, l);
        case EPI_SVREM: return with_potential<EPI_SVREM, float>(pot, l);
        case EPI_SVRG: return with_potential<EPI_SVRG, float>(pot, l);
        case EPI_ANCHOR: return with_potential<EPI_ANCHOR, float>(pot, l);
        case EPI_SAGA:
            return bf ? with_potential<EPI_SAGA, __nv_bfloat16>(pot, l) : with_potential<EPI_SAGA, float>(pot, l);
        case EPI_SAGA_INIT:
            return bf ? with_potential<EPI_SAGA_INIT, __nv_bfloat16>(pot, l)
                      : with_potential<EPI_SAGA_INIT, float>(pot, l);
        case EPI_SGA: return with_potential<EPI_SGA, float>(pot, l);
        case EPI_SEM: return with_potential<EPI_SEM, float>(pot, l);
        case EPI_SEM_INIT: return with_potential<EPI_SEM_INIT, float>(pot, l);
        case EPI_SAGAEM: return with_potential<EPI_SAGAEM, float>(pot, l);
        case EPI_SAGAEM_INIT: return with_potential<EPI_SAGAEM_INIT, float>(pot, l);
        default: return set_error(PET_ERR_INVALID, "back: unknown epilogue");
    }
}

}  // namespace

}  // namespace petvr
