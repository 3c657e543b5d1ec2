// Plain-FP32 (CUDA-core) Born contractions with fused Green's-function synthesis.
//
// Adjoint and Gauss-Newton diagonal (per frequency w, S = W o R):
//   U[e][x] = sum_r S[e][r] conj(G_r(x)),   g(x) = w^2 sum_e conj(G_e(x)) U[e][x]
//   V[e][x] = sum_r W[e][r] |G_r(x)|^2,     H(x) = w^4 sum_e |G_e(x)|^2 V[e][x]
// One CTA owns a tile of 32 pixels: it synthesises G_t(x) for every element
// and the tile's pixels into shared memory (Eqs. 4-5), runs both
// contractions over r with S and W streamed through shared memory in chunks,
// and reduces over e in a fixed order, so g and H never need U or V in HBM
// and every pixel's result is independent of scheduling.
//
// Forward: d[e][r] = w^2 sum_x G_e(x) G_r(x) m(x), symmetric in (e, r).  Split-K
// over pixel chunks: CTA (tile pair, chunk) accumulates a 64x64 block of the
// upper triangle; a second kernel sums the chunk partials in a fixed order
// and mirrors the block.
#include "rb_internal.cuh"

namespace {

constexpr int AP = 32;     // pixels per adjoint tile
constexpr int AT = 256;    // threads per adjoint CTA: 8 pixel groups x 32 element groups
constexpr int RC = 8;      // r-chunk of S / W staged in shared memory
constexpr int RCP = RC + 1;  // padded row (conflict-free reads by the 4 element rows of a warp)

// G tile synthesis: Gs[t][p] for t < n_elem, p < AP (zero beyond npix).
__device__ __forceinline__ void synth_tile(const GeoDev& G, const rb_cell* __restrict__ tables, const float* __restrict__ c,
                                           const FreqC& F, int p0, float2* Gs) {
    const int n = G.n_elem;
    for (int idx = threadIdx.x; idx < n * AP; idx += blockDim.x) {
        const int t = idx / AP, p = idx % AP;
        const int pix = p0 + p;
        float2 v = make_float2(0.f, 0.f);
        if (pix < G.npix) {
            const rb_cell rec = tables[(size_t)t * G.npix + pix];
            const int ix = pix % G.nx, iy = pix / G.nx;
            if (rec.tkey != RB_HOLE) {
                DF ex, ey;
                elem_pos(G, t, ex, ey);
                const DF dist = pixel_elem_dist(G, ix, iy, ex, ey);
                v = green_eval(rec, __ldg(c + pix), dist, F, G.j_floor);
            }
        }
        Gs[t * AP + p] = v;
    }
}

template <int EPT>
__global__ void __launch_bounds__(AT) k_adjoint_simt(GeoDev G, const rb_cell* __restrict__ tables, const float* __restrict__ c,
                                                     FreqSet F, const float2* __restrict__ resid, const uint8_t* __restrict__ w,
                                                     float2* __restrict__ g_out, float* __restrict__ h_out,
                                                     float* __restrict__ gsum, float* __restrict__ hsum,
                                                     uint32_t* __restrict__ counters) {
    extern __shared__ float4 smem4[];
    const int n = G.n_elem;
    float2* Gs = (float2*)smem4;                 // [n][AP]
    float2* Ss = Gs + (size_t)n * AP;            // [n][RCP]
    float* Ws = (float*)(Ss + (size_t)n * RCP);  // [n][RCP]
    float* red = (float*)Ss;                     // [32][AP][3], reuses the S/W staging after the r loop
    const int tx = threadIdx.x & 7;              // pixel group: pixels tx*4 .. tx*4+3
    const int ty = threadIdx.x >> 3;             // element group: e = ty + 32 i, i < EPT
    const int p0 = blockIdx.x * AP;
    float acc_g = 0.f, acc_h = 0.f;              // running sums over w (threads < AP)

    for (int fw = 0; fw < F.n; ++fw) {
        const FreqC& fc = F.f[fw];
        const float2* Rw = resid + (size_t)fw * n * n;
        const uint8_t* Ww = w + (size_t)fw * n * n;
        __syncthreads();
        synth_tile(G, tables, c, fc, p0, Gs);
        float ur[EPT][4], ui[EPT][4], vv[EPT][4];
#pragma unroll
        for (int i = 0; i < EPT; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ur[i][j] = ui[i][j] = vv[i][j] = 0.f;
        for (int r0 = 0; r0 < n; r0 += RC) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < n * RC; idx += blockDim.x) {
                const int e = idx / RC, rr = idx % RC;
                const int r = r0 + rr;
                float2 s = make_float2(0.f, 0.f);
                float wv = 0.f;
                if (r < n) {
                    const uint8_t wb = Ww[(size_t)e * n + r];
                    if (wb) {
                        s = Rw[(size_t)e * n + r];
                        wv = 1.f;
                    }
                }
                Ss[e * RCP + rr] = s;
                Ws[e * RCP + rr] = wv;
            }
            __syncthreads();
            const int rmax = min(RC, n - r0);
            for (int rr = 0; rr < rmax; ++rr) {
                const float4* gp = (const float4*)(Gs + (size_t)(r0 + rr) * AP + tx * 4);
                const float4 g01 = gp[0], g23 = gp[1];
                const float br[4] = {g01.x, g01.z, g23.x, g23.z};
                const float bi[4] = {-g01.y, -g01.w, -g23.y, -g23.w};   // conj(G_r)
                float a2[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) a2[j] = br[j] * br[j] + bi[j] * bi[j];
#pragma unroll
                for (int i = 0; i < EPT; ++i) {
                    const int e = ty + 32 * i;
                    const float2 s = (e < n) ? Ss[e * RCP + rr] : make_float2(0.f, 0.f);
                    const float wv = (e < n) ? Ws[e * RCP + rr] : 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        ur[i][j] = fmaf(s.x, br[j], fmaf(-s.y, bi[j], ur[i][j]));
                        ui[i][j] = fmaf(s.x, bi[j], fmaf(s.y, br[j], ui[i][j]));
                        vv[i][j] = fmaf(wv, a2[j], vv[i][j]);
                    }
                }
            }
        }
        // epilogue: partial sums over this thread's elements, then a fixed-order reduction over ty
        float pg_r[4], pg_i[4], ph[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) pg_r[j] = pg_i[j] = ph[j] = 0.f;
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            const int e = ty + 32 * i;
            if (e >= n) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 ge = Gs[(size_t)e * AP + tx * 4 + j];
                const float cr = ge.x, ci = -ge.y;   // conj(G_e)
                pg_r[j] += cr * ur[i][j] - ci * ui[i][j];
                pg_i[j] += cr * ui[i][j] + ci * ur[i][j];
                ph[j] += (ge.x * ge.x + ge.y * ge.y) * vv[i][j];
            }
        }
        __syncthreads();   // every thread is done with the S/W staging that red reuses
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = tx * 4 + j;
            red[(ty * AP + p) * 3 + 0] = pg_r[j];
            red[(ty * AP + p) * 3 + 1] = pg_i[j];
            red[(ty * AP + p) * 3 + 2] = ph[j];
        }
        __syncthreads();
        if (threadIdx.x < AP) {
            const int p = threadIdx.x;
            float sr = 0.f, si = 0.f, sh = 0.f;
            for (int q = 0; q < 32; ++q) {
                sr += red[(q * AP + p) * 3 + 0];
                si += red[(q * AP + p) * 3 + 1];
                sh += red[(q * AP + p) * 3 + 2];
            }
            sr *= fc.w2;
            si *= fc.w2;
            sh *= fc.w4;
            const int pix = p0 + p;
            if (pix < G.npix) {
                if (g_out) g_out[(size_t)fw * G.npix + pix] = make_float2(sr, si);
                if (h_out) h_out[(size_t)fw * G.npix + pix] = sh;
            }
            acc_g += sr;
            acc_h += sh;
        }
    }
    if (threadIdx.x < AP) {
        const int pix = p0 + threadIdx.x;
        if (pix < G.npix) {
            if (gsum) gsum[pix] = acc_g;
            if (hsum) hsum[pix] = acc_h;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
constexpr int FT = 64;      // element tile
constexpr int FP = 32;      // pixels per sub-tile
constexpr int FTHR = 256;   // 16 x 16 threads, 4 x 4 complex outputs each

__global__ void __launch_bounds__(FTHR) k_forward_simt(GeoDev G, const rb_cell* __restrict__ tables, const float* __restrict__ c,
                                                       FreqC F, const float* __restrict__ m, float2* __restrict__ partial,
                                                       int n_chunks) {
    __shared__ float2 Ae[FP][FT + 1];   // G_e(x) m(x), transposed [p][e] (padded rows)
    __shared__ float2 Br[FP][FT + 1];   // G_r(x)
    const int n = G.n_elem;
    const int nt = (n + FT - 1) / FT;
    // decode the upper-triangular tile pair from blockIdx.x
    int pair = blockIdx.x, te = 0;
    while (pair >= nt - te) { pair -= nt - te; ++te; }
    const int tr = te + pair;
    const int chunk = blockIdx.y;
    const int pix_per = (G.npix + n_chunks - 1) / n_chunks;
    const int pbeg = chunk * pix_per, pend = min(G.npix, pbeg + pix_per);
    const int e0 = te * FT, r0 = tr * FT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.f;

    for (int ps = pbeg; ps < pend; ps += FP) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < 2 * FT * FP; idx += FTHR) {
            const int which = idx / (FT * FP);
            const int rem = idx % (FT * FP);
            const int tl = rem / FP, p = rem % FP;
            const int t = (which == 0 ? e0 : r0) + tl;
            const int pix = ps + p;
            float2 v = make_float2(0.f, 0.f);
            if (t < n && pix < pend) {
                const rb_cell rec = tables[(size_t)t * G.npix + pix];
                if (rec.tkey != RB_HOLE) {
                    const int ix = pix % G.nx, iy = pix / G.nx;
                    DF ex, ey;
                    elem_pos(G, t, ex, ey);
                    v = green_eval(rec, __ldg(c + pix), pixel_elem_dist(G, ix, iy, ex, ey), F, G.j_floor);
                    if (which == 0) {
                        const float mv = __ldg(m + pix);
                        v.x *= mv;
                        v.y *= mv;
                    }
                }
            }
            if (which == 0) Ae[p][tl] = v; else Br[p][tl] = v;
        }
        __syncthreads();
        const int np = min(FP, pend - ps);
        for (int p = 0; p < np; ++p) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = Ae[p][ty * 4 + i];
                b[i] = Br[p][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ar[i][j] = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, ar[i][j]));
                    ai[i][j] = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, ai[i][j]));
                }
        }
    }
    // partial[chunk][e][r] for this block (upper-triangle tile pairs only)
    float2* out = partial + (size_t)chunk * n * n;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = e0 + ty * 4 + i, r = r0 + tx * 4 + j;
            if (e < n && r < n) out[(size_t)e * n + r] = make_float2(ar[i][j], ai[i][j]);
        }
}

// d[e][r] = w^2 sum_chunk partial (fixed order); lower triangle mirrored from the
// upper tiles; optional sum of W |d|^2 into per-block partials.
__global__ void k_forward_reduce(GeoDev G, FreqC F, const float2* __restrict__ partial, int n_chunks,
                                 float2* __restrict__ d_out, const uint8_t* __restrict__ w, double* __restrict__ den_part) {
    const int n = G.n_elem;
    const long long total = (long long)n * n;
    double acc = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(j / n), r = (int)(j % n);
        // source entry in the upper triangle of tiles
        const int te = e / FT, tr = r / FT;
        const long long src = (te <= tr) ? j : (long long)r * n + e;
        float sr = 0.f, si = 0.f;
        for (int ch = 0; ch < n_chunks; ++ch) {
            const float2 v = partial[(size_t)ch * total + src];
            sr += v.x;
            si += v.y;
        }
        sr *= F.w2;
        si *= F.w2;
        if (d_out) d_out[j] = make_float2(sr, si);
        if (w && w[j]) acc += (double)sr * sr + (double)si * si;
    }
    if (den_part) {
        __shared__ double sred[256];
        sred[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sred[threadIdx.x] += sred[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) den_part[blockIdx.x] = sred[0];
    }
}

// Green's functions written out, g[w][t][pixel] (tests and users who want G itself).
__global__ void k_green_out(GeoDev G, const rb_cell* __restrict__ tables, const float* __restrict__ c, FreqSet F,
                            float2* __restrict__ g) {
    const long long total = (long long)G.n_elem * G.npix;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(j / G.npix), pix = (int)(j % G.npix);
        const rb_cell rec = tables[j];
        const int ix = pix % G.nx, iy = pix / G.nx;
        DF ex, ey;
        elem_pos(G, t, ex, ey);
        const DF dist = pixel_elem_dist(G, ix, iy, ex, ey);
        const float cv = __ldg(c + pix);
        for (int w = 0; w < F.n; ++w) g[(size_t)w * total + j] = green_eval(rec, cv, dist, F.f[w], G.j_floor);
    }
}

}  // namespace

cudaError_t launch_green_out(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F, float2* g_out,
                             cudaStream_t s) {
    const long long total = (long long)G.n_elem * G.npix;
    long long blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_green_out<<<(int)blocks, 256, 0, s>>>(G, tables, c, F, g_out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_simt(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F,
                                const float2* resid, const uint8_t* w, float2* g_out, float* h_out, float* gsum,
                                float* hsum, uint32_t* counters, cudaStream_t s) {
    const int n = G.n_elem;
    size_t stage = (size_t)n * RCP * (sizeof(float2) + sizeof(float));
    const size_t redb = (size_t)32 * AP * 3 * sizeof(float);
    if (stage < redb) stage = redb;
    const size_t sm = (size_t)n * AP * sizeof(float2) + stage;
    const int blocks = (G.npix + AP - 1) / AP;
    const int ept = (n + 31) / 32;
#define RB_LAUNCH_ADJ(E)                                                                                          \
    do {                                                                                                          \
        cudaError_t e_ = cudaFuncSetAttribute(k_adjoint_simt<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                              (int)sm);                                                           \
        if (e_ != cudaSuccess) return e_;                                                                         \
        k_adjoint_simt<E><<<blocks, AT, sm, s>>>(G, tables, c, F, resid, w, g_out, h_out, gsum, hsum, counters);   \
    } while (0)
    if (ept <= 2) RB_LAUNCH_ADJ(2);
    else if (ept <= 4) RB_LAUNCH_ADJ(4);
    else if (ept <= 8) RB_LAUNCH_ADJ(8);
    else if (ept <= 16) RB_LAUNCH_ADJ(16);
    else return cudaErrorInvalidValue;
#undef RB_LAUNCH_ADJ
    return cudaGetLastError();
}

// the adjoint holds a 32-pixel tile of G for every element in shared memory and gives
// each lane at most 16 elements: rings of up to 512 elements
bool simt_adjoint_supported(int n_elem) { return n_elem >= 2 && (n_elem + 31) / 32 <= 16; }

int rb_fwd_chunks_for(int npix) {
    int ch = (npix + 2047) / 2048;
    if (ch < 1) ch = 1;
    if (ch > 128) ch = 128;
    return ch;
}

cudaError_t launch_forward_simt(const GeoDev& G, const rb_cell* tables, const float* c, const FreqC& F, const float* m,
                                float2* partial, int n_chunks, cudaStream_t s) {
    const int nt = (G.n_elem + FT - 1) / FT;
    dim3 grid(nt * (nt + 1) / 2, n_chunks);
    k_forward_simt<<<grid, FTHR, 0, s>>>(G, tables, c, F, m, partial, n_chunks);
    return cudaGetLastError();
}

cudaError_t launch_forward_reduce(const GeoDev& G, const FreqC& F, const float2* partial, int n_chunks, float2* d_out,
                                  const uint8_t* w, double* den_part, cudaStream_t s) {
    k_forward_reduce<<<256, 256, 0, s>>>(G, F, partial, n_chunks, d_out, w, den_part);
    return cudaGetLastError();
}
