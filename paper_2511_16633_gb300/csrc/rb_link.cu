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

// Traveltime of receiver dr's bracket by interval i, in explicitly rounded steps so
// that every evaluation of the same bracket gives the same bits.
__device__ __forceinline__ double bracket_T(double chord_t, double a, double b, double thr, double tri, double tri1,
                                            double* lam_out) {
    const double den = __dsub_rn(b, a);
    const double lam = den != 0.0 ? __ddiv_rn(__dsub_rn(thr, a), den) : 0.0;
    *lam_out = lam;
    return __dadd_rn(chord_t, __dadd_rn(__dmul_rn(__dsub_rn(1.0, lam), tri), __dmul_rn(lam, tri1)));
}

// Order-preserving map of a double to uint64 (for the first-arrival minimum).
__device__ __forceinline__ unsigned long long d2key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// One CTA per emitter e.  The end angles of its fan go to shared memory; then each
// thread takes ray intervals (i, i + 1) and visits only the receivers whose angle
// lies in that interval's range, so the work is O(n_rays + brackets) rather than
// O(n_rays x n_elem).  The first arrival per receiver is the minimum of an
// order-preserving 64-bit traveltime key (shared-memory atomic min), ties to the
// smallest interval index in a second pass, which reproduces a sequential scan
// over i that keeps the first strictly smaller T.
__global__ void __launch_bounds__(256) k_link(GeoDev G, const float* __restrict__ c, const rb_ray_end* __restrict__ ends,
                                              FreqSet F, float2* __restrict__ p_out, uint8_t* __restrict__ linked,
                                              LinkRec* __restrict__ lrec) {
    extern __shared__ unsigned char smem[];
    const int n = G.n_rays, N = G.n_elem;
    double* th = (double*)smem;                             // [n]
    double* tr = th + n;                                    // [n]
    double* cht = tr + n;                                   // [N] chord / c_ref per receiver offset dr
    unsigned long long* best = (unsigned long long*)(cht + N);   // [N] first-arrival key per dr
    float* qq = (float*)(best + N);                         // [n]
    float* ll = qq + n;                                     // [n]
    int* kk = (int*)(ll + n);                               // [n]
    int* ok = kk + n;                                       // [n]
    int* bi = ok + n;                                       // [N] winning interval per dr
    const int e = blockIdx.x;
    const double two_pi = 2.0 * RB_PI_D;
    const double phi_e = two_pi * (double)e / (double)N;
    double xe, ye;
    sincos(phi_e, &ye, &xe);
    xe *= G.R_d;
    ye *= G.R_d;
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
    for (int dr = threadIdx.x; dr < N; dr += blockDim.x) {
        const int r = (e + dr) % N;
        double xr, yr;
        sincos(two_pi * (double)r / (double)N, &yr, &xr);
        xr *= G.R_d;
        yr *= G.R_d;
        cht[dr] = sqrt((xr - xe) * (xr - xe) + (yr - ye) * (yr - ye)) / G.c_ref_d;
        best[dr] = ~0ull;
        bi[dr] = 0x7fffffff;
    }
    __syncthreads();
    const double dN = (double)N / two_pi;
    // pass 1: first-arrival key per receiver; pass 2: smallest interval with that key
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) {
            if (!ok[i] || !ok[i + 1]) continue;
            const double a = th[i], b = th[i + 1];
            if (fabs(b - a) > RB_PI_D) continue;
            const double lo = fmin(a, b), hi = fmax(a, b);
            // receiver offsets whose angle 2 pi dr / N can lie in [lo, hi] (one spare each side)
            const int d0 = max(0, (int)floor(lo * dN) - 1), d1 = min(N - 1, (int)ceil(hi * dN) + 1);
            for (int dr = d0; dr <= d1; ++dr) {
                const double thr = two_pi * (double)dr / (double)N;
                if (thr < lo || thr > hi) continue;
                double lam;
                const unsigned long long key = d2key(bracket_T(cht[dr], a, b, thr, tr[i], tr[i + 1], &lam));
                if (pass == 0) atomicMin(&best[dr], key);
                else if (key == best[dr]) atomicMin(&bi[dr], i);
            }
        }
        __syncthreads();
    }
    for (int dr = threadIdx.x; dr < N; dr += blockDim.x) {
        const int r = (e + dr) % N;
        const size_t o = (size_t)e * N + r;
        const int bsel = bi[dr];
        if (linked) linked[o] = bsel != 0x7fffffff ? 1 : 0;
        if (bsel == 0x7fffffff) {
            if (lrec) lrec[o] = LinkRec{0.0, -1, 0.f};
            for (int w = 0; w < F.n; ++w) p_out[(size_t)w * N * N + o] = make_float2(0.f, 0.f);
            continue;
        }
        const double thr = two_pi * (double)dr / (double)N;
        double bestLam;
        const double bestT = bracket_T(cht[dr], th[bsel], th[bsel + 1], thr, tr[bsel], tr[bsel + 1], &bestLam);
        if (lrec) lrec[o] = LinkRec{bestT, bsel, (float)bestLam};
        if (F.n == 0) continue;
        double xr, yr;
        sincos(two_pi * (double)r / (double)N, &yr, &xr);
        xr *= G.R_d;
        yr *= G.R_d;
        const float lf = (float)bestLam;
        const float q = (1.f - lf) * qq[bsel] + lf * qq[bsel + 1];
        const float L = (1.f - lf) * ll[bsel] + lf * ll[bsel + 1];
        const int kap = bestLam <= 0.5 ? kk[bsel] : kk[bsel + 1];
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
            p_out[(size_t)w * N * N + o] = make_float2(amp * co, amp * s);
        }
    }
}

// Workspace of the outlier selection (rb_sel_bytes): a 12-bit histogram of the top
// digit of the keys, a few scalars, then the compacted candidates of one bucket.
constexpr int SEL_THREADS = 1024;
constexpr int SEL_BINS = 4096;          // top 12 bits
constexpr int SEL_CAP = 12288;          // compacted candidates (96 KB of shared memory)
constexpr int SEL_BLOCKS = 64;          // CTAs of the grid-wide passes
struct SelHdr {
    uint32_t hist[SEL_BINS];
    uint32_t n_cand;                    // candidates found in the bucket (may exceed SEL_CAP)
    uint32_t pad[3];
    unsigned long long thr;             // selected threshold (keys below it keep W = 1)
};

// R = p_ray - p_obs in place; keys for the outlier selection; kept count; the
// histogram of the keys' top 12 bits (per CTA in shared memory, then added to
// the global one, which the caller zeroed).
__global__ void __launch_bounds__(SEL_THREADS) k_residual_keys(GeoDev G, int n_freq, const float2* __restrict__ p_obs,
                                                               float2* __restrict__ r, const uint8_t* __restrict__ linked,
                                                               uint64_t* __restrict__ keys, uint32_t* __restrict__ counters,
                                                               SelHdr* __restrict__ sel) {
    __shared__ uint32_t hist[SEL_BINS];
    for (int b = threadIdx.x; b < SEL_BINS; b += blockDim.x) hist[b] = 0;
    __syncthreads();
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
            atomicAdd(&hist[key >> 52], 1u);
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
    __syncthreads();
    for (int b = threadIdx.x; b < SEL_BINS; b += blockDim.x)
        if (hist[b]) atomicAdd(&sel->hist[b], hist[b]);
}

// Exact selection of the k-th largest non-zero 64-bit key, k = floor(frac * kept)
// (keys are distinct: the low word is the entry index); W = 1 for the non-zero keys
// below it.  Grid-wide passes: the histogram above picks the top-digit bucket that
// holds the k-th largest (k_sel_compact, every CTA computes the same bucket by a
// block-wide suffix scan), the bucket's keys are compacted, one CTA resolves the
// remaining 52 bits by 8-bit radix passes in shared memory (k_sel_final; a bucket
// larger than the shared buffer is resolved by passes over the global keys), and
// the weights are written grid-wide (k_sel_write).

// Bucket d (top 12 bits) holding the k-th largest key and the rank rem of that key
// within it, from the global histogram; called by all SEL_THREADS threads of a CTA.
__device__ void sel_bucket(const uint32_t* __restrict__ ghist, long long k, int* d_out, long long* rem_out) {
    __shared__ long long warp_tot[SEL_THREADS / 32];
    __shared__ int s_d;
    __shared__ long long s_rem;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    uint32_t h4[4];
    long long own = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h4[q] = ghist[4 * t + q];
        own += h4[q];
    }
    // inclusive suffix sum over threads (thread t covers bins 4t .. 4t + 3): scan in
    // reverse thread order within warps, then over the warps
    long long v = own;
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o < 32) v += u;
    }
    if (lane == 0) warp_tot[wid] = v;
    if (t == 0) s_d = -1;
    __syncthreads();
    long long above = 0;
    for (int w2 = wid + 1; w2 < SEL_THREADS / 32; ++w2) above += warp_tot[w2];
    const long long incl = v + above, excl = incl - own;
    if (excl < k && k <= incl) {
        long long rem = k - excl;
        int d = 4 * t;
        for (int q = 3; q >= 0; --q) {
            if ((long long)h4[q] >= rem) {
                d = 4 * t + q;
                break;
            }
            rem -= h4[q];
        }
        s_d = d;
        s_rem = rem;
    }
    __syncthreads();
    *d_out = s_d;
    *rem_out = s_rem;
    __syncthreads();
}

__global__ void __launch_bounds__(SEL_THREADS) k_sel_compact(int n_total, double frac, const uint64_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ counters,
                                                             SelHdr* __restrict__ sel, uint64_t* __restrict__ cand) {
    const long long k = (long long)floor(frac * (double)counters[CNT_KEPT]);
    if (k <= 0) return;
    int d;
    long long rem;
    sel_bucket(sel->hist, k, &d, &rem);
    if (d < 0) return;
    const uint64_t top = (uint64_t)d << 52;
    const int lane = threadIdx.x & 31;
    // warp-uniform loop bounds: every lane takes part in the ballot
    for (int j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < n_total; j0 += gridDim.x * blockDim.x) {
        const int j = j0 + lane;
        const uint64_t key = j < n_total ? keys[j] : 0ull;
        const bool hit = key != 0 && (key & (0xfffull << 52)) == top;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (!m) continue;
        uint32_t base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(&sel->n_cand, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (hit) {
            const uint32_t idx = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
            if (idx < (uint32_t)SEL_CAP) cand[idx] = key;
        }
    }
}

// Resolve bits 51..0 of the k-th largest key within the bucket given by prefix /
// rem from `src` (n entries; shared or global), 8 bits per pass (4 in the last).
__device__ uint64_t sel_resolve(const uint64_t* src, int n, uint64_t prefix, long long rem, uint32_t* hist) {
    __shared__ uint64_t s_prefix;
    __shared__ long long s_rem;
    if (threadIdx.x == 0) {
        s_prefix = prefix;
        s_rem = rem;
    }
    uint64_t mask = 0xfffull << 52;
    for (int shift = 44; shift >= -4; shift -= 8) {
        const int sh = shift < 0 ? 0 : shift;
        const int bits = shift < 0 ? 4 : 8;          // last pass: bits 3..0
        const uint64_t dm = (1ull << bits) - 1;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint64_t pre = s_prefix;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const uint64_t key = src[j];
            if (key != 0 && (key & mask) == pre) atomicAdd(&hist[(key >> sh) & dm], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long r = s_rem;
            int d = (int)dm;
            for (; d > 0; --d) {
                if ((long long)hist[d] >= r) break;
                r -= hist[d];
            }
            s_rem = r;
            s_prefix = pre | ((uint64_t)d << sh);
        }
        mask |= dm << sh;
        __syncthreads();
    }
    return s_prefix;
}

__global__ void __launch_bounds__(SEL_THREADS) k_sel_final(int n_total, double frac, const uint64_t* __restrict__ keys,
                                                           uint32_t* __restrict__ counters, SelHdr* __restrict__ sel,
                                                           const uint64_t* __restrict__ cand) {
    extern __shared__ uint64_t scand[];          // [SEL_CAP]
    __shared__ uint32_t hist[256];
    const long long k = (long long)floor(frac * (double)counters[CNT_KEPT]);
    uint64_t thr = ~0ull;   // nothing zeroed
    if (k > 0) {
        int d;
        long long rem;
        sel_bucket(sel->hist, k, &d, &rem);
        const int nc = (int)sel->n_cand;
        if (d < 0) {
            // fewer non-zero keys than k (not reachable: k < kept): nothing is zeroed
        } else if (nc <= SEL_CAP) {
            for (int j = threadIdx.x; j < nc; j += blockDim.x) scand[j] = cand[j];
            __syncthreads();
            thr = sel_resolve(scand, nc, (uint64_t)d << 52, rem, hist);
        } else {
            thr = sel_resolve(keys, n_total, (uint64_t)d << 52, rem, hist);
        }
    }
    if (threadIdx.x == 0) {
        sel->thr = thr;
        counters[CNT_ZEROED] = (uint32_t)(k > 0 ? k : 0);
    }
}

__global__ void k_sel_write(int n_total, const uint64_t* __restrict__ keys, const SelHdr* __restrict__ sel,
                            uint8_t* __restrict__ w) {
    const uint64_t thr = sel->thr;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_total; j += gridDim.x * blockDim.x) {
        const uint64_t key = keys[j];
        w[j] = (key != 0 && key < thr) ? 1 : 0;
    }
}

}  // namespace

cudaError_t launch_link(const GeoDev& G, const float* c, const rb_ray_end* ends, const FreqSet& F, float2* p_out,
                        uint8_t* linked, cudaStream_t s, LinkRec* lrec) {
    if (G.n_rays > LINK_MAX_RAYS) return cudaErrorInvalidValue;
    const size_t sm = (size_t)G.n_rays * (8 + 8 + 4 + 4 + 4 + 4) + (size_t)G.n_elem * (8 + 8 + 4);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_link, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_link<<<G.n_elem, 256, sm, s>>>(G, c, ends, F, p_out, linked, lrec);
    return cudaGetLastError();
}

size_t rb_sel_bytes() { return sizeof(SelHdr) + (size_t)SEL_CAP * sizeof(uint64_t); }

cudaError_t launch_residual_keys(const GeoDev& G, int n_freq, const float2* p_obs, float2* r_inout,
                                 const uint8_t* linked, uint64_t* keys, uint32_t* counters, void* sel_ws,
                                 cudaStream_t s) {
    SelHdr* sel = (SelHdr*)sel_ws;
    cudaError_t e = cudaMemsetAsync(sel, 0, sizeof(SelHdr), s);
    if (e != cudaSuccess) return e;
    const long long total = (long long)n_freq * G.n_elem * G.n_elem;
    long long blocks = (total + SEL_THREADS - 1) / SEL_THREADS;
    if (blocks > SEL_BLOCKS) blocks = SEL_BLOCKS;
    k_residual_keys<<<(int)blocks, SEL_THREADS, 0, s>>>(G, n_freq, p_obs, r_inout, linked, keys, counters, sel);
    return cudaGetLastError();
}

cudaError_t launch_outlier_select(int n_total, double frac, const uint64_t* keys, uint32_t* counters, uint8_t* w,
                                  void* sel_ws, cudaStream_t s) {
    SelHdr* sel = (SelHdr*)sel_ws;
    uint64_t* cand = (uint64_t*)((char*)sel_ws + sizeof(SelHdr));
    long long blocks = ((long long)n_total + SEL_THREADS - 1) / SEL_THREADS;
    if (blocks > SEL_BLOCKS) blocks = SEL_BLOCKS;
    if (blocks < 1) blocks = 1;
    k_sel_compact<<<(int)blocks, SEL_THREADS, 0, s>>>(n_total, frac, keys, counters, sel, cand);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int sm = SEL_CAP * (int)sizeof(uint64_t);
    e = cudaFuncSetAttribute(k_sel_final, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_sel_final<<<1, SEL_THREADS, sm, s>>>(n_total, frac, keys, counters, sel, cand);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long wb = ((long long)n_total + 255) / 256;
    if (wb > 1024) wb = 1024;
    if (wb < 1) wb = 1;
    k_sel_write<<<(int)wb, 256, 0, s>>>(n_total, keys, sel, w);
    return cudaGetLastError();
}
