// Forward projectors for volumes (K1): slice stacks (nz independent slices
// sharing one 2-D geometry) and multi-ring scanners (fully 3-D lines of
// response through a voxel volume).  They write the same ratio /
// log-likelihood outputs as the single-slice kernels (forward.cu); their back
// projections are in volume_back.cu.
#include "epilogue.cuh"

namespace petvr {

namespace {

// Slice-stack forward: the geometry is shared by every slice.  A warp takes
// one ray and a window of 8 ZW consecutive slices; its lanes are kStackChunks
// band chunks x 8 z-lanes, and z-lane l carries slices l, l + 8, ... of the
// window, so each load instruction reads 8 consecutive floats of a pixel's
// slice column per chunk ([iy][ix][z] layout: coalesced).  The band geometry
// is evaluated once per band: in each batch of 8 bands of a chunk, z-lane l
// evaluates band kbase + l and the chunk's other lanes take its pixel offset
// and weights by shuffles.  Bands are added in order within a chunk (w0 piece,
// then w1 piece) and the chunk sums are combined by xor-shuffles in a fixed
// order, so the result is deterministic.
template <int MODE, bool LL, int ZW>
__global__ void __launch_bounds__(kBlock) forward_stack_kernel(const FwdArgs a) {
    const RayRange rr = ray_range(a);
    // 32-bit index arithmetic: images and sinograms are below 2^31 elements (checked at plan time)
    const int n_rays = (rr.v_end - rr.v_begin) * a.nb;
    const int n_win = (a.nz + 8 * ZW - 1) / (8 * ZW);
    const int lane = threadIdx.x & 31;
    const int zl = lane & 7;                              // z-lane
    const int chunk = lane >> 3;                          // band chunk (kStackChunks = 4 per warp)
    const unsigned gmask = 0xffu << (8 * chunk);          // the chunk's 8 lanes
    const long long wid = (long long)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    const int ray = (int)min(wid / n_win, (long long)n_rays);
    const int win = (int)(wid % n_win);
    const bool live = ray < n_rays;                       // the same for the whole warp
    const int z0 = win * 8 * ZW + zl;                     // this lane's first slice
    const int n_zi = live ? min(ZW, max(0, (a.nz - z0 + 7) / 8)) : 0;   // slices this lane carries

    float acc[ZW];
#pragma unroll
    for (int i = 0; i < ZW; ++i) acc[i] = 0.0f;
    if (live) {
        const int p = rr.v_begin + ray / a.nb;
        const int j = ray % a.nb;
        const int v = __ldg(a.order + p);
        const ViewParams vp = a.views[v];
        const float2 u = __ldg(a.uc + v * a.nb + j);
        const int n_major = vp.col ? a.nx : a.ny;
        const int n_minor = vp.col ? a.ny : a.nx;
        const float hm = 0.5f * (float)n_major;
        int k_lo, k_hi;
        band_range(vp, u.x + u.y, n_major, n_minor, k_lo, k_hi);
        const int per = (n_major + kStackChunks - 1) / kStackChunks;
        const int kb = max(k_lo, chunk * per);
        const int ke = min(k_hi, (chunk + 1) * per);
        const int s_major = vp.col ? 1 : a.nx;            // pixel strides
        const int s_minor = vp.col ? a.nx : 1;
        const int ui = (int)u.x + (n_minor >> 1);         // pixel index of fractional position 0
        const float *img = a.img + z0;
        for (int kbase = kb; kbase < ke; kbase += 8) {    // the same trip count for the chunk's 8 lanes
            const int k = kbase + zl;
            int n0 = 0;
            float c0 = 0.0f, c1 = 0.0f;
            if (k < ke) {
                const float kc = (float)k - hm;
                float fl, w0, w1;
                band_split(vp, band_point(vp, u.y, kc), band_point(vp, u.y, kc + 1.0f), fl, w0, w1);
                const int m0 = (int)fl + ui;
                n0 = k * s_major + m0 * s_minor;
                c0 = (unsigned)m0 < (unsigned)n_minor ? w0 : 0.0f;
                c1 = w1 > 0.0f && (unsigned)(m0 + 1) < (unsigned)n_minor ? w1 : 0.0f;
            }
            const int nbands = min(8, ke - kbase);
            for (int b = 0; b < nbands; ++b) {
                const int nb0 = __shfl_sync(gmask, n0, b, 8);
                const float w0b = __shfl_sync(gmask, c0, b, 8);
                const float w1b = __shfl_sync(gmask, c1, b, 8);
                if (w0b != 0.0f) {
                    const float *px = img + nb0 * a.nz;
#pragma unroll
                    for (int i = 0; i < ZW; ++i)
                        if (i < n_zi) acc[i] = fmaf(w0b, __ldg(px + 8 * i), acc[i]);
                }
                if (w1b != 0.0f) {
                    const float *px = img + (nb0 + s_minor) * a.nz;
#pragma unroll
                    for (int i = 0; i < ZW; ++i)
                        if (i < n_zi) acc[i] = fmaf(w1b, __ldg(px + 8 * i), acc[i]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ZW; ++i) {
        acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 8);
        acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 16);
    }

    // every chunk holds the totals now; in round e chunk c finishes slice
    // i = kStackChunks e + c, so the warp runs each round's epilogue once
    double ll = 0.0;
#pragma unroll
    for (int e = 0; e < (ZW + kStackChunks - 1) / kStackChunks; ++e) {
        float val = acc[e * kStackChunks];
#pragma unroll
        for (int c = 1; c < kStackChunks; ++c)
            if (e * kStackChunks + c < ZW && chunk == c) val = acc[e * kStackChunks + c];
        const int i = e * kStackChunks + chunk;
        if (i >= ZW || i >= n_zi) continue;
        const int idx = ray * a.nz + z0 + 8 * i;
        const long long gi = rr.off + idx;
        const float yhat = val + (a.w ? __ldg(a.w + gi) : a.w_scalar);
        if (MODE == FWD_YHAT) a.out[idx] = yhat;
        if (MODE == FWD_RATIO || LL) {
            const float g = __ldg(a.g + gi);
            if (MODE == FWD_RATIO) a.out[idx] = (yhat != 0.0f) ? g / yhat : 0.0f;
            if (LL) {
                if (yhat > 0.0f) {
                    // per-ray term with an FP32 log (GB300's FP64 pipe is too slow for a
                    // log per ray; the term's error, ~g ulp(log yhat), is far below the
                    // FP32 rounding of yhat itself), reduced in FP64
                    ll += (g > 0.0f ? (double)g * (double)logf(yhat) : 0.0) - (double)yhat;
                } else if (g > 0.0f) {
                    ll = -(double)INFINITY;            // log of a nonpositive mean: Phi = -inf
                    if (a.status) atomicExch(a.status, (int)PET_ERR_NUMERIC);
                } else {
                    ll += -(double)yhat;
                }
            }
        }
    }
    if (LL) {
        __shared__ double red[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ll;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
#pragma unroll
            for (int i = 0; i < kBlock / 32; ++i) sum += red[i];
            a.ll_partials[blockIdx.x] = sum;
        }
    }
}

// Multi-ring forward: CH consecutive lanes per ray, each walking one chunk of
// the ray's bands (chunks aligned to the same bands for every ray, so
// neighbouring rays read the same image rows) and carrying the sums of all
// P ring pairs of the ray in registers: the transaxial work of a band is done
// once for its P lines.  Every band piece is spread over the layers each
// line's axial range crosses (piece_fraction / piece_zeta / layer_fraction,
// shared with the back projection).  The chunk sums are combined by
// xor-shuffles in a fixed order; lane c writes the lines c, c + CH, ...
template <int MODE, bool LL, int CH, int P>
__global__ void __launch_bounds__(kBlock) ring_forward_kernel(const FwdArgs a) {
    const RayRange rr = ray_range(a);
    // 32-bit index arithmetic: sinograms and images are below 2^31 elements (checked at plan time)
    const int n_rays = (rr.v_end - rr.v_begin) * a.nb;
    const long long gtid = (long long)blockIdx.x * kBlock + threadIdx.x;
    const int chunk = (int)(gtid % CH);
    const int ray = (int)min(gtid / CH, (long long)n_rays);
    const bool live = ray < n_rays;
    float acc[P];
#pragma unroll
    for (int pr = 0; pr < P; ++pr) acc[pr] = 0.0f;
    if (live) {
        const int q = rr.v_begin + ray / a.nb;
        const int j = ray % a.nb;
        const int v = __ldg(a.order + q);
        const ViewParams vp = a.views[v];
        const float2 u = __ldg(a.uc + v * a.nb + j);
        const float4 *lzr = a.lz + (v * a.nb + j) * P;
        const int n_major = vp.col ? a.nx : a.ny;
        const int n_minor = vp.col ? a.ny : a.nx;
        const float hm = 0.5f * (float)n_major;
        const int ui = (int)u.x + (n_minor >> 1);
        const int s_major = vp.col ? 1 : a.nx;           // pixel strides
        const int s_minor = vp.col ? a.nx : 1;
        const int L = a.layers;
        int k_lo, k_hi;
        band_range(vp, u.x + u.y, n_major, n_minor, k_lo, k_hi);
        const int per = (n_major + CH - 1) / CH;
        const int kb = max(k_lo, chunk * per);
        const int ke = min(k_hi, (chunk + 1) * per);
        float kc = (float)kb - hm;
        float va = band_point(vp, u.y, kc);
        for (int k = kb; k < ke; ++k) {
            const float vb = band_point(vp, u.y, kc + 1.0f);
            float fl, w0, w1;
            band_split(vp, va, vb, fl, w0, w1);
            const int m0 = (int)fl + ui;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int m = m0 + side;
                const float w = side ? w1 : w0;
                if (!(w > 0.0f) || (unsigned)m >= (unsigned)n_minor) continue;
                float f_lo, f_hi;
                piece_fraction(vp, w0, w1, side == 1, f_lo, f_hi);
                const float *colp = a.img + (k * s_major + m * s_minor) * L;     // < 2^31 (plan check)
#pragma unroll
                for (int pr = 0; pr < P; ++pr) {
                    const float4 lz = __ldg(lzr + pr);
                    const float za = piece_zeta(lz, kc, f_lo), zb = piece_zeta(lz, kc, f_hi);
                    const float wl = w * lz.z;
                    const int il = max(0, (int)floorf(fminf(za, zb)));
                    const int ih = min(L - 1, (int)floorf(fmaxf(za, zb)));
                    for (int iz = il; iz <= ih; ++iz) {
                        const float fr = layer_fraction(za, zb, iz);
                        if (fr > 0.0f) acc[pr] = fmaf(wl * fr, __ldg(colp + iz), acc[pr]);
                    }
                }
            }
            va = vb;
            kc += 1.0f;
        }
    }
#pragma unroll
    for (int pr = 0; pr < P; ++pr)
#pragma unroll
        for (int o = CH / 2; o > 0; o >>= 1) acc[pr] += __shfl_xor_sync(0xffffffffu, acc[pr], o);
    double ll = 0.0;
    if (live) {
        // round e: chunk lane c finishes line pr = CH e + c, so the warp runs
        // each round's epilogue once
#pragma unroll
        for (int e = 0; e < (P + CH - 1) / CH; ++e) {
            float val = acc[e * CH];
#pragma unroll
            for (int c = 1; c < CH && e * CH + c < P; ++c)
                if (chunk == c) val = acc[e * CH + c];
            const int pr = e * CH + chunk;
            if (pr >= P) continue;
            const int idx = ray * P + pr;
            const long long gi = rr.off + idx;
            const float yhat = val + (a.w ? __ldg(a.w + gi) : a.w_scalar);
            if (MODE == FWD_YHAT) a.out[idx] = yhat;
            if (MODE == FWD_RATIO || LL) {
                const float g = __ldg(a.g + gi);
                if (MODE == FWD_RATIO) a.out[idx] = (yhat != 0.0f) ? g / yhat : 0.0f;
                if (LL) {
                    if (yhat > 0.0f) {
                        ll += (g > 0.0f ? (double)g * (double)logf(yhat) : 0.0) - (double)yhat;
                    } else if (g > 0.0f) {
                        ll = -(double)INFINITY;        // log of a nonpositive mean: Phi = -inf
                        if (a.status) atomicExch(a.status, (int)PET_ERR_NUMERIC);
                    } else {
                        ll += -(double)yhat;
                    }
                }
            }
        }
    }
    if (LL) {
        __shared__ double red[kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ll;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
#pragma unroll
            for (int i = 0; i < kBlock / 32; ++i) sum += red[i];
            a.ll_partials[blockIdx.x] = sum;
        }
    }
}

// Nonzeros of the multi-ring lines of a view range: (piece, layer) pairs of
// positive weight, with the projector's own geometry (one thread per line).
__global__ void __launch_bounds__(kBlock) ring_count_nnz_kernel(const FwdArgs a, unsigned long long *count) {
    const int P = a.nz;
    const long long n_lor = (long long)(a.v_end - a.v_begin) * a.nb * P;
    const long long tid = (long long)blockIdx.x * kBlock + threadIdx.x;
    unsigned long long c = 0;
    if (tid < n_lor) {
        const int pr = (int)(tid % P);
        const long long ray = tid / P;
        const int v = a.order[a.v_begin + (int)(ray / a.nb)];
        const int j = (int)(ray % a.nb);
        const ViewParams vp = a.views[v];
        const float2 u = a.uc[(long long)v * a.nb + j];
        const float4 lz = a.lz[((long long)v * a.nb + j) * P + pr];
        const int n_major = vp.col ? a.nx : a.ny;
        const int n_minor = vp.col ? a.ny : a.nx;
        const int ui = (int)u.x + (n_minor >> 1);
        float kc = -0.5f * (float)n_major;
        float va = band_point(vp, u.y, kc);
        for (int k = 0; k < n_major; ++k) {
            const float vb = band_point(vp, u.y, kc + 1.0f);
            float fl, w0, w1;
            band_split(vp, va, vb, fl, w0, w1);
            const int m0 = (int)fl + ui;
            for (int side = 0; side < 2; ++side) {
                const float w = side ? w1 : w0;
                if (!(w > 0.0f) || (unsigned)(m0 + side) >= (unsigned)n_minor) continue;
                float f_lo, f_hi;
                piece_fraction(vp, w0, w1, side == 1, f_lo, f_hi);
                const float za = piece_zeta(lz, kc, f_lo), zb = piece_zeta(lz, kc, f_hi);
                const int il = max(0, (int)floorf(fminf(za, zb)));
                const int ih = min(a.layers - 1, (int)floorf(fmaxf(za, zb)));
                for (int iz = il; iz <= ih; ++iz) c += layer_fraction(za, zb, iz) > 0.0f ? 1 : 0;
            }
            va = vb;
            kc += 1.0f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

template <int CH, int P>
pet_status dispatch_ring_p(const FwdArgs &a, int mode, bool ll, int blocks, cudaStream_t s) {
    if (mode == FWD_YHAT && !ll)
        ring_forward_kernel<FWD_YHAT, false, CH, P><<<blocks, kBlock, 0, s>>>(a);
    else if (mode == FWD_RATIO && !ll)
        ring_forward_kernel<FWD_RATIO, false, CH, P><<<blocks, kBlock, 0, s>>>(a);
    else if (mode == FWD_RATIO && ll)
        ring_forward_kernel<FWD_RATIO, true, CH, P><<<blocks, kBlock, 0, s>>>(a);
    else if (mode == FWD_NONE && ll)
        ring_forward_kernel<FWD_NONE, true, CH, P><<<blocks, kBlock, 0, s>>>(a);
    else
        return set_error(PET_ERR_INVALID, "forward: unsupported mode");
    return check_launch("ring_forward_kernel");
}

template <int CH>
pet_status dispatch_ring(const FwdArgs &a, int mode, bool ll, int blocks, cudaStream_t s) {
    switch (a.nz) {                                      // ring pairs: n_rings^2, n_rings <= 4
        case 1: return dispatch_ring_p<CH, 1>(a, mode, ll, blocks, s);
        case 4: return dispatch_ring_p<CH, 4>(a, mode, ll, blocks, s);
        case 9: return dispatch_ring_p<CH, 9>(a, mode, ll, blocks, s);
        case 16: return dispatch_ring_p<CH, 16>(a, mode, ll, blocks, s);
        default: return set_error(PET_ERR_INVALID, "forward: unsupported number of ring pairs");
    }
}

template <int ZW>
pet_status dispatch_stack_zw(const FwdArgs &a, int mode, bool ll, int blocks, cudaStream_t s) {
    if (mode == FWD_YHAT && !ll)
        forward_stack_kernel<FWD_YHAT, false, ZW><<<blocks, kBlock, 0, s>>>(a);
    else if (mode == FWD_RATIO && !ll)
        forward_stack_kernel<FWD_RATIO, false, ZW><<<blocks, kBlock, 0, s>>>(a);
    else if (mode == FWD_RATIO && ll)
        forward_stack_kernel<FWD_RATIO, true, ZW><<<blocks, kBlock, 0, s>>>(a);
    else if (mode == FWD_NONE && ll)
        forward_stack_kernel<FWD_NONE, true, ZW><<<blocks, kBlock, 0, s>>>(a);
    else
        return set_error(PET_ERR_INVALID, "forward: unsupported mode");
    return check_launch("forward_stack_kernel");
}

pet_status dispatch_stack(const FwdArgs &a, int mode, bool ll, int blocks, cudaStream_t s) {
    switch (stack_lane_slices(a.nz)) {
        case 2: return dispatch_stack_zw<2>(a, mode, ll, blocks, s);
        case 4: return dispatch_stack_zw<4>(a, mode, ll, blocks, s);
        case 6: return dispatch_stack_zw<6>(a, mode, ll, blocks, s);
        default: return dispatch_stack_zw<8>(a, mode, ll, blocks, s);
    }
}

}  // namespace

pet_status launch_forward_volume(const FwdArgs &a, int mode, bool ll, int group, int blocks, cudaStream_t s) {
    if (a.lz) {
        switch (group) {
            case 8: return dispatch_ring<8>(a, mode, ll, blocks, s);
            case 16: return dispatch_ring<16>(a, mode, ll, blocks, s);
            case 32: return dispatch_ring<32>(a, mode, ll, blocks, s);
            default: return set_error(PET_ERR_INVALID, "forward: unsupported band chunk count");
        }
    }
    if (group != kStackChunks) return set_error(PET_ERR_INVALID, "forward: slice stacks use 4 band chunks");
    return dispatch_stack(a, mode, ll, blocks, s);
}

pet_status launch_count_nnz_ring(const FwdArgs &a, unsigned long long *d_count, cudaStream_t s) {
    const long long n_lor = (long long)(a.v_end - a.v_begin) * a.nb * a.nz;
    if (n_lor == 0) return PET_OK;
    ring_count_nnz_kernel<<<(unsigned)((n_lor + kBlock - 1) / kBlock), kBlock, 0, s>>>(a, d_count);
    return check_launch("ring_count_nnz_kernel");
}

}  // namespace petvr
