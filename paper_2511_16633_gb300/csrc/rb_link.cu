// Ray linking, residuals and data-space weights.
//
// Ray linking (the ray-model data p(c) of Eq. 8): fan e's rays end on the
// ring at angles vartheta_i = atan2(end) - phi_e (wrapped to [0, 2 pi)); the
// neighbouring pair (i, i+1), both ended on the ring and less than pi apart,
// brackets receiver r when vartheta_r lies between its end angles.  T (as the
// residual against the chord's water time), Q and L are interpolated
// linearly in angle and kappa comes from the nearer ray (the lower one on a
// tie); the smallest T over all brackets wins (ties: lowest i).  p_ray is the
// Green's function of Eqs. 4-5 at the receiver, with c sampled bilinearly.
//
// Data weights (Sec. 4.1): receivers on the opposite ~75 % of the ring
// (circular index distance >= ceil(N/8)), linked pairs only, then per
// frequency set the floor(frac * kept) entries of largest |R| are zeroed,
// ties to the smallest flat index (w, e, r).  The selection is an exact
// radix select on 64-bit keys (|R|^2 bits, complemented index), so it is
// deterministic and identical to a sort.
#include "rb_internal.cuh"

namespace {

constexpr int LINK_MAX_RAYS = 4096;

__device__ __forceinline__ float bilinear_c(const GeoDev& G, const float* __restrict__ c, float x, float y) {
    float u = fminf(fmaxf(x * G.inv_h + G.cxg, 0.f), (float)(G.nx - 1));
    float v = fminf(fmaxf(y * G.inv_h + G.cyg, 0.f), (float)(G.ny - 1));
    const int i0 = min((int)u, G.nx - 2), j0 = min((int)v, G.ny - 2);
    const float fu = u - (float)i0, fv = v - (float)j0;
    const float* p = c + (size_t)j0 * G.nx + i0;
    return (1.f - fu) * (1.f - fv) * p[0] + fu * (1.f - fv) * p[1] + (1.f - fu) * fv * p[G.nx] + fu * fv * p[G.nx + 1];
}

__global__ void __launch_bounds__(256) k_link(GeoDev G, const float* __restrict__ c, const rb_ray_end* __restrict__ ends,
                                              FreqSet F, float2* __restrict__ p_out, uint8_t* __restrict__ linked) {
    extern __shared__ unsigned char smem[];
    const int n = G.n_rays;
    double* th = (double*)smem;            // [n]
    double* tr = th + n;                   // [n]
    float* qq = (float*)(tr + n);          // [n]
    float* ll = qq + n;                    // [n]
    int* kk = (int*)(ll + n);              // [n]
    int* ok = kk + n;                      // [n]
    const int e = blockIdx.x;
    const double two_pi = 2.0 * RB_PI_D;
    const double phi_e = two_pi * (double)e / (double)G.n_elem;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const rb_ray_end E = ends[(size_t)e * n + i];
        double a = atan2(E.y, E.x) - phi_e;
        a = fmod(a, two_pi);
        if (a < 0.0) a += two_pi;
        if (a >= two_pi) a -= two_pi;
        th[i] = a;
        tr[i] = E.t_res;
        qq[i] = E.q;
        ll[i] = E.l;
        kk[i] = E.kappa;
        ok[i] = E.n_vert > 0;
    }
    __syncthreads();
    double xe, ye;
    sincos(phi_e, &ye, &xe);
    xe *= G.R_d;
    ye *= G.R_d;
    for (int r = threadIdx.x; r < G.n_elem; r += blockDim.x) {
        const int dr = ((r - e) % G.n_elem + G.n_elem) % G.n_elem;
        const double thr = two_pi * (double)dr / (double)G.n_elem;
        double xr, yr;
        sincos(two_pi * (double)r / (double)G.n_elem, &yr, &xr);
        xr *= G.R_d;
        yr *= G.R_d;
        const double chord = sqrt((xr - xe) * (xr - xe) + (yr - ye) * (yr - ye));
        double bestT = 1e300, bestLam = 0.0;
        int best = -1;
        for (int i = 0; i + 1 < n; ++i) {
            if (!ok[i] || !ok[i + 1]) continue;
            const double a = th[i], b = th[i + 1];
            if (fabs(b - a) > RB_PI_D) continue;
            const double lo = fmin(a, b), hi = fmax(a, b);
            if (thr < lo || thr > hi) continue;
            const double den = b - a;
            const double lam = den != 0.0 ? (thr - a) / den : 0.0;
            const double T = chord / G.c_ref_d + (1.0 - lam) * tr[i] + lam * tr[i + 1];
            if (T < bestT) {
                bestT = T;
                bestLam = lam;
                best = i;
            }
        }
        const size_t o = (size_t)e * G.n_elem + r;
        if (linked) linked[o] = best >= 0 ? 1 : 0;
        if (best < 0) {
            for (int w = 0; w < F.n; ++w) p_out[(size_t)w * G.n_elem * G.n_elem + o] = make_float2(0.f, 0.f);
            continue;
        }
        const float lf = (float)bestLam;
        const float q = (1.f - lf) * qq[best] + lf * qq[best + 1];
        const float L = (1.f - lf) * ll[best] + lf * ll[best + 1];
        const int kap = bestLam <= 0.5 ? kk[best] : kk[best + 1];
        const float crx = bilinear_c(G, c, (float)xr, (float)yr);
        const float J = fmaxf(fabsf(q), G.j_floor);
        for (int w = 0; w < F.n; ++w) {
            const FreqC& fc = F.f[w];
            const double fT = fc.f_d * bestT;
            double cyc = fT - rint(fT);
            cyc += (double)fc.disp_cyc * (double)L + 0.125 - 0.25 * (double)(kap & 3);
            cyc -= rint(cyc);
            float s, co;
            sincospif(2.0f * (float)cyc, &s, &co);
            const float amp = sqrtf(crx / (8.0f * RB_PI_F * J)) * fc.w_isqrt * expf(-fc.a_abs * L);
            p_out[(size_t)w * G.n_elem * G.n_elem + o] = make_float2(amp * co, amp * s);
        }
    }
}

// R = p_ray - p_obs in place; keys for the outlier selection; kept count.
__global__ void k_residual_keys(GeoDev G, int n_freq, const float2* __restrict__ p_obs, float2* __restrict__ r,
                                const uint8_t* __restrict__ linked, uint64_t* __restrict__ keys,
                                uint32_t* __restrict__ counters) {
    const int N = G.n_elem;
    const long long total = (long long)n_freq * N * N;
    const int min_sep = (N + 7) / 8;
    uint32_t kept = 0, unlinked = 0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
        const int er = (int)(j % ((long long)N * N));
        const int e = er / N, rr = er % N;
        int d = abs(e - rr);
        d = min(d, N - d);
        const bool in_mask = d >= min_sep;
        const bool lk = linked[er] != 0;
        const float2 p = r[j], o = p_obs[j];
        const float2 R = make_float2(p.x - o.x, p.y - o.y);
        r[j] = R;
        uint64_t key = 0;
        if (in_mask && lk) {
            const float m2 = R.x * R.x + R.y * R.y;
            key = ((uint64_t)__float_as_uint(m2) << 32) | (uint64_t)(0xffffffffu - (uint32_t)j);
            ++kept;
        }
        if (in_mask && !lk && j < (long long)N * N) ++unlinked;
        keys[j] = key;
    }
    // warp-aggregated counters
    for (int o = 16; o > 0; o >>= 1) {
        kept += __shfl_down_sync(0xffffffffu, kept, o);
        unlinked += __shfl_down_sync(0xffffffffu, unlinked, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (kept) atomicAdd(counters + CNT_KEPT, kept);
        if (unlinked) atomicAdd(counters + CNT_UNLINKED, unlinked);
    }
}

// Exact selection of the k-th largest non-zero 64-bit key (keys are distinct: the
// low word is the entry index), then W = 1 for the non-zero keys below it.  One CTA:
// a 12-bit histogram of the top digit over all keys picks the bucket that holds the
// k-th largest; that bucket's keys are compacted into shared memory and the
// remaining 52 bits are resolved there by 8-bit radix passes.  A bucket larger than
// the shared buffer falls back to radix passes over the global keys.
constexpr int SEL_THREADS = 1024;
constexpr int SEL_BINS = 4096;          // top 12 bits
constexpr int SEL_CAP = 12288;          // compacted candidates (96 KB of shared memory)

// Find, among bins [0, nb) counted in hist (largest digit = highest bin), the bin
// that holds the rem-th largest key; returns it and leaves in *rem the rank within it.
__device__ int sel_pick(const uint32_t* hist, int nb, long long* rem_io) {
    // sequential from the top; called by one thread on at most 4096 bins
    long long rem = *rem_io;
    int d = nb - 1;
    for (; d > 0; --d) {
        if ((long long)hist[d] >= rem) break;
        rem -= hist[d];
    }
    *rem_io = rem;
    return d;
}

__global__ void __launch_bounds__(SEL_THREADS) k_outlier_select(int n_total, double frac, const uint64_t* __restrict__ keys,
                                                                uint32_t* __restrict__ counters, uint8_t* __restrict__ w) {
    extern __shared__ uint64_t cand[];           // [SEL_CAP]
    __shared__ uint32_t hist[SEL_BINS];
    __shared__ uint64_t s_prefix;
    __shared__ long long s_rem;
    __shared__ int s_d, s_nc;
    const uint32_t kept = counters[CNT_KEPT];
    const long long k = (long long)floor(frac * (double)kept);
    uint64_t thr = ~0ull;   // nothing zeroed
    if (k > 0) {
        for (int b = threadIdx.x; b < SEL_BINS; b += blockDim.x) hist[b] = 0;
        if (threadIdx.x == 0) {
            s_rem = k;
            s_nc = 0;
        }
        __syncthreads();
        // four independent loads in flight per thread and iteration
        for (int j0 = threadIdx.x; j0 < n_total; j0 += 4 * blockDim.x) {
            uint64_t kk[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = j0 + t * blockDim.x;
                kk[t] = j < n_total ? keys[j] : 0ull;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (kk[t] != 0) atomicAdd(&hist[kk[t] >> 52], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long rem = s_rem;
            s_d = sel_pick(hist, SEL_BINS, &rem);
            s_rem = rem;
            s_prefix = (uint64_t)s_d << 52;
        }
        __syncthreads();
        const int nb = (int)hist[s_d];
        uint64_t mask = 0xfffull << 52;
        if (nb <= SEL_CAP) {
            // compact the bucket, then 8-bit passes over bits 51..0 in shared memory
            const uint64_t top = s_prefix;
            for (int j0 = threadIdx.x; j0 < n_total; j0 += 4 * blockDim.x) {
                uint64_t kk[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = j0 + t * blockDim.x;
                    kk[t] = j < n_total ? keys[j] : 0ull;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (kk[t] != 0 && (kk[t] & mask) == top) cand[atomicAdd(&s_nc, 1)] = kk[t];
            }
            __syncthreads();
            const int nc = s_nc;
            for (int shift = 44; shift >= -4; shift -= 8) {
                const int sh = shift < 0 ? 0 : shift;
                const int bits = shift < 0 ? 4 : 8;          // last pass: bits 3..0
                const uint64_t dm = (1ull << bits) - 1;
                for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
                __syncthreads();
                const uint64_t pre = s_prefix;
                for (int j = threadIdx.x; j < nc; j += blockDim.x) {
                    const uint64_t key = cand[j];
                    if ((key & mask) == pre) atomicAdd(&hist[(key >> sh) & dm], 1u);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    long long rem = s_rem;
                    const int d = sel_pick(hist, (int)dm + 1, &rem);
                    s_rem = rem;
                    s_prefix = pre | ((uint64_t)d << sh);
                }
                mask |= dm << sh;
                __syncthreads();
            }
        } else {
            for (int shift = 44; shift >= -4; shift -= 8) {
                const int sh = shift < 0 ? 0 : shift;
                const int bits = shift < 0 ? 4 : 8;
                const uint64_t dm = (1ull << bits) - 1;
                for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
                __syncthreads();
                const uint64_t pre = s_prefix;
                for (int j = threadIdx.x; j < n_total; j += blockDim.x) {
                    const uint64_t key = keys[j];
                    if (key != 0 && (key & mask) == pre) atomicAdd(&hist[(key >> sh) & dm], 1u);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    long long rem = s_rem;
                    const int d = sel_pick(hist, (int)dm + 1, &rem);
                    s_rem = rem;
                    s_prefix = pre | ((uint64_t)d << sh);
                }
                mask |= dm << sh;
                __syncthreads();
            }
        }
        thr = s_prefix;
    }
    for (int j0 = threadIdx.x; j0 < n_total; j0 += 4 * blockDim.x) {
        uint64_t kk[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = j0 + t * blockDim.x;
            kk[t] = j < n_total ? keys[j] : 0ull;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = j0 + t * blockDim.x;
            if (j < n_total) w[j] = (kk[t] != 0 && kk[t] < thr) ? 1 : 0;
        }
    }
    if (threadIdx.x == 0) counters[CNT_ZEROED] = (uint32_t)k;
}

}  // namespace

cudaError_t launch_link(const GeoDev& G, const float* c, const rb_ray_end* ends, const FreqSet& F, float2* p_out,
                        uint8_t* linked, cudaStream_t s) {
    if (G.n_rays > LINK_MAX_RAYS) return cudaErrorInvalidValue;
    const size_t sm = (size_t)G.n_rays * (8 + 8 + 4 + 4 + 4 + 4);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_link, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_link<<<G.n_elem, 256, sm, s>>>(G, c, ends, F, p_out, linked);
    return cudaGetLastError();
}

cudaError_t launch_residual_keys(const GeoDev& G, int n_freq, const float2* p_obs, float2* r_inout,
                                 const uint8_t* linked, uint64_t* keys, uint32_t* counters, cudaStream_t s) {
    const long long total = (long long)n_freq * G.n_elem * G.n_elem;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_residual_keys<<<blocks, 256, 0, s>>>(G, n_freq, p_obs, r_inout, linked, keys, counters);
    return cudaGetLastError();
}

cudaError_t launch_outlier_select(int n_total, double frac, const uint64_t* keys, const uint32_t* /*counters*/,
                                  uint8_t* w, uint32_t* counters_out, cudaStream_t s) {
    const int sm = SEL_CAP * (int)sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(k_outlier_select, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_outlier_select<<<1, SEL_THREADS, sm, s>>>(n_total, frac, keys, counters_out, w);
    return cudaGetLastError();
}
