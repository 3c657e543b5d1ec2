// Tensor-core (tcgen05, BF16 x3 split products, FP32 accumulation in TMEM) Born
// adjoint and Gauss-Newton Hessian diagonal with fused Green's-function synthesis.
//
// Per frequency w and tile of 128 pixels x (the MMA's M rows):
//   U[x][e']  = sum_k' A[x][k'] B[e'][k'],   k' = 2r + {0: Re, 1: Im}
//     A[x][2r] = Re G_r(x), A[x][2r+1] = -Im G_r(x)           (conj G, synthesised)
//     e' < n:  B = (Re S[e][r], -Im S[e][r])  ->  U = Re (S conj G)[e]
//     e' >= n: B = (Im S[e][r],  Re S[e][r])  ->  U = Im (S conj G)[e]
//   g(x) = w^2 sum_e conj(G_e(x)) U_e(x),  S = W o R
//   V[x][e]   = sum_r |G_r(x)|^2 W[e][r],    H(x) = w^4 sum_e |G_e(x)|^2 V[x][e]
// Each operand is split into bf16 hi + lo and the products hi*hi + hi*lo + lo*hi
// (U) or hi*W + lo*W (V, W is exact in bf16) accumulate in fp32 in TMEM, which
// keeps ~2^-16 relative accuracy per product.  The epilogue uses the exact fp32
// G values, kept per CTA in a small L2-resident scratch while the K loop streams
// bf16 chunks of A through shared memory.
#include "rb_internal.cuh"
#include "rb_tc.cuh"

namespace {

constexpr int TP = 128;                 // pixels per tile = MMA M
constexpr int NTHR = 128;               // threads per CTA: thread = pixel = TMEM lane
constexpr uint32_t kMaxTries = 1u << 22; // mbarrier polls before giving up (each poll suspends briefly)

// ---------------------------------------------------------------------------
// B operand images for one frequency, chunked by 32 columns of K in the
// core-matrix layout of rb_tc.cuh.
//   bu: [kc = 2n/32][hi|lo][2n rows x 32]   (2n rows = e', K = 2n)
//   bw: [kc = n/32][n rows x 32]            (W, exact)
// ---------------------------------------------------------------------------
__global__ void k_prep_b(int n, const float2* __restrict__ R, const uint8_t* __restrict__ W,
                         __nv_bfloat16* __restrict__ bu, __nv_bfloat16* __restrict__ bw) {
    const int n2 = 2 * n;
    const size_t img_u = (size_t)n2 * 32;  // bf16 per hi or lo image of one chunk
    const long long total_u = (long long)n2 * n2;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total_u;
         j += (long long)gridDim.x * blockDim.x) {
        const int ep = (int)(j / n2), kp = (int)(j % n2);
        const int r = kp >> 1, part = kp & 1;
        const int e = ep % n, blk = ep / n;
        float2 s = make_float2(0.f, 0.f);
        if (W[(size_t)e * n + r]) s = R[(size_t)e * n + r];
        float v;
        if (blk == 0) v = part == 0 ? s.x : -s.y;
        else v = part == 0 ? s.y : s.x;
        __nv_bfloat16 hi, lo;
        tc::split_bf16(v, hi, lo);
        const int kc = kp >> 5, kk = kp & 31;
        const size_t base = (size_t)kc * 2 * img_u;
        const uint32_t off = tc::chunk_offset((uint32_t)ep, (uint32_t)kk) / 2;
        bu[base + off] = hi;
        bu[base + img_u + off] = lo;
    }
    const long long total_w = (long long)n * n;
    const size_t img_w = (size_t)n * 32;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total_w;
         j += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(j / n), r = (int)(j % n);
        const int kc = r >> 5, kk = r & 31;
        bw[(size_t)kc * img_w + tc::chunk_offset((uint32_t)e, (uint32_t)kk) / 2] =
            __float2bfloat16_rn(W[(size_t)e * n + r] ? 1.f : 0.f);
    }
}

struct TcArgs {
    GeoDev G;
    FreqSet F;
    const rb_cell* tables;
    const float* c;
    const __nv_bfloat16* bu;   // [n_freq][image]
    const __nv_bfloat16* bw;   // [n_freq][image]
    size_t bu_stride, bw_stride;  // bf16 elements per frequency
    float2* gscr;              // [gridDim.x][n][TP] exact G per CTA
    float2* g_out;             // [n_freq][npix] or null
    float* h_out;              // [n_freq][npix] or null
    float* gsum;               // [npix] or null (sum over w of Re g)
    float* hsum;               // [npix] or null
    uint32_t* counters;
    int n_tiles;
    uint32_t tmem_cols;
};

// cooperative 16-byte copy of `bytes` (multiple of 16) from global to shared
__device__ __forceinline__ void copy_chunk(void* dst, const void* src, int bytes) {
    const uint4* s = (const uint4*)src;
    uint4* d = (uint4*)dst;
    for (int i = threadIdx.x; i < bytes / 16; i += NTHR) d[i] = __ldg(s + i);
}

}  // namespace

namespace {

// Synthesise this thread's pixel row of one A chunk: G_r for r in [r0, r0 + 16),
// (Re, -Im) split into bf16 hi/lo, stored in the core-matrix layout; exact values to gs.
__device__ __forceinline__ void synth_a_chunk(const TcArgs& A, const FreqC& fc, int r0, int px, bool valid, int ix,
                                              int iy, float c_px, float2* gs, unsigned char* sa_hi,
                                              unsigned char* sa_lo) {
    const GeoDev& G = A.G;
    uint32_t whi[16], wlo[16];
#pragma unroll 4
    for (int j = 0; j < 16; ++j) {
        const int r = r0 + j;
        float2 g = make_float2(0.f, 0.f);
        if (valid) {
            const rb_cell rec = A.tables[(size_t)r * G.npix + px];
            if (rec.tkey != RB_HOLE) {
                const DF ex = df_from_double(G.elem_xy[2 * r]), ey = df_from_double(G.elem_xy[2 * r + 1]);
                g = green_eval(rec, c_px, pixel_elem_dist(G, ix, iy, ex, ey), fc, G.j_floor);
            }
        }
        gs[(size_t)r * TP + threadIdx.x] = g;
        __nv_bfloat16 h0, l0, h1, l1;
        tc::split_bf16(g.x, h0, l0);
        tc::split_bf16(-g.y, h1, l1);
        whi[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        wlo[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const uint32_t row = (uint32_t)threadIdx.x;
#pragma unroll
    for (int kg = 0; kg < 4; ++kg) {
        const uint32_t off = tc::chunk_offset(row, 8u * kg);
        *(uint4*)(sa_hi + off) = make_uint4(whi[4 * kg], whi[4 * kg + 1], whi[4 * kg + 2], whi[4 * kg + 3]);
        *(uint4*)(sa_lo + off) = make_uint4(wlo[4 * kg], wlo[4 * kg + 1], wlo[4 * kg + 2], wlo[4 * kg + 3]);
    }
}

// |G_r(x)|^2 for r in [r0, r0 + 32) from the exact values, split into bf16 hi/lo.
__device__ __forceinline__ void synth_a2_chunk(int r0, const float2* gs, unsigned char* sa_hi, unsigned char* sa_lo) {
    uint32_t whi[16], wlo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float2 g0 = gs[(size_t)(r0 + 2 * j) * TP + threadIdx.x];
        const float2 g1 = gs[(size_t)(r0 + 2 * j + 1) * TP + threadIdx.x];
        __nv_bfloat16 h0, l0, h1, l1;
        tc::split_bf16(g0.x * g0.x + g0.y * g0.y, h0, l0);
        tc::split_bf16(g1.x * g1.x + g1.y * g1.y, h1, l1);
        whi[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        wlo[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const uint32_t row = (uint32_t)threadIdx.x;
#pragma unroll
    for (int kg = 0; kg < 4; ++kg) {
        const uint32_t off = tc::chunk_offset(row, 8u * kg);
        *(uint4*)(sa_hi + off) = make_uint4(whi[4 * kg], whi[4 * kg + 1], whi[4 * kg + 2], whi[4 * kg + 3]);
        *(uint4*)(sa_lo + off) = make_uint4(wlo[4 * kg], wlo[4 * kg + 1], wlo[4 * kg + 2], wlo[4 * kg + 3]);
    }
}

constexpr uint32_t OFF_AHI = 0, OFF_ALO = 8192, OFF_B = 16384;

__global__ void __launch_bounds__(NTHR, 1) k_adjoint_tc(TcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    const GeoDev& G = A.G;
    const int n = G.n_elem, n2 = 2 * n;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char* sa_hi = smem + OFF_AHI;
    unsigned char* sa_lo = smem + OFF_ALO;
    unsigned char* sb_hi = smem + OFF_B;
    unsigned char* sb_lo = smem + OFF_B + (size_t)n2 * 64;
    const uint32_t mbar = tc::smem_u32(&s_mbar);
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), A.tmem_cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const int nbk = n2 > 256 ? 2 : 1;
    const int nb_u = n2 / nbk;
    const uint32_t id_u = tc::idesc_bf16_f32(128, (uint32_t)nb_u);
    const uint32_t id_v = tc::idesc_bf16_f32(128, (uint32_t)n);
    const size_t img_u = (size_t)n2 * 32, img_w = (size_t)n * 32;   // bf16 elements
    float2* gs = A.gscr + (size_t)blockIdx.x * n * TP;
    uint32_t phase = 0;
    bool ok = true;

    for (int tile = blockIdx.x; tile < A.n_tiles && ok; tile += gridDim.x) {
        const int px = tile * TP + tid;
        const bool valid = px < G.npix;
        const int ix = valid ? px % G.nx : 0, iy = valid ? px / G.nx : 0;
        const float c_px = valid ? __ldg(A.c + px) : 0.f;
        float acc_g = 0.f, acc_h = 0.f;
        for (int fw = 0; fw < A.F.n && ok; ++fw) {
            const FreqC& fc = A.F.f[fw];
            const __nv_bfloat16* bu = A.bu + (size_t)fw * A.bu_stride;
            const __nv_bfloat16* bw = A.bw + (size_t)fw * A.bw_stride;
            // ---- U = A B^T over K' = 2n, chunks of 32 ----
            for (int kc = 0; kc < n2 / 32 && ok; ++kc) {
                synth_a_chunk(A, fc, kc * 16, px, valid, ix, iy, c_px, gs, sa_hi, sa_lo);
                copy_chunk(sb_hi, bu + (size_t)kc * 2 * img_u, n2 * 64);
                copy_chunk(sb_lo, bu + (size_t)kc * 2 * img_u + img_u, n2 * 64);
                tc::fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after();
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ah = tc::sdesc(tc::smem_u32(sa_hi) + 256u * ks, 128, 512);
                        const uint64_t al = tc::sdesc(tc::smem_u32(sa_lo) + 256u * ks, 128, 512);
                        for (int nb = 0; nb < nbk; ++nb) {
                            const uint32_t boff = (uint32_t)(nb * nb_u / 8) * 512u + 256u * ks;
                            const uint64_t bh = tc::sdesc(tc::smem_u32(sb_hi) + boff, 128, 512);
                            const uint64_t bl = tc::sdesc(tc::smem_u32(sb_lo) + boff, 128, 512);
                            const uint32_t d = tmem + (uint32_t)(nb * nb_u);
                            tc::mma_bf16(d, ah, bh, id_u, (kc > 0 || ks > 0) ? 1u : 0u);
                            tc::mma_bf16(d, ah, bl, id_u, 1u);
                            tc::mma_bf16(d, al, bh, id_u, 1u);
                        }
                    }
                    tc::commit(mbar);
                }
                ok = __syncthreads_and(tc::mbar_wait(mbar, phase, kMaxTries) ? 1 : 0) != 0;
                phase ^= 1u;
            }
            if (!ok) break;
            tc::fence_after();
            float gr = 0.f, gi = 0.f;
            for (int cb = 0; cb < n2; cb += 32) {
                float v[32];
                tc::tmem_ld32(tmem + lane_off + (uint32_t)cb, v);
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const int ep = cb + j;
                    const int e = ep < n ? ep : ep - n;
                    const float2 ge = gs[(size_t)e * TP + tid];
                    if (ep < n) {
                        gr = fmaf(ge.x, v[j], gr);
                        gi = fmaf(-ge.y, v[j], gi);
                    } else {
                        gr = fmaf(ge.y, v[j], gr);
                        gi = fmaf(ge.x, v[j], gi);
                    }
                }
            }
            gr *= fc.w2;
            gi *= fc.w2;
            if (valid && A.g_out) A.g_out[(size_t)fw * G.npix + px] = make_float2(gr, gi);
            acc_g += gr;
            tc::fence_before();
            __syncthreads();
            // ---- V = A2 W^T over K = n, chunks of 32 (accumulator reuses the first n columns) ----
            for (int kc = 0; kc < n / 32 && ok; ++kc) {
                synth_a2_chunk(kc * 32, gs, sa_hi, sa_lo);
                copy_chunk(sb_hi, bw + (size_t)kc * img_w, n * 64);
                tc::fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after();
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ah = tc::sdesc(tc::smem_u32(sa_hi) + 256u * ks, 128, 512);
                        const uint64_t al = tc::sdesc(tc::smem_u32(sa_lo) + 256u * ks, 128, 512);
                        const uint64_t b = tc::sdesc(tc::smem_u32(sb_hi) + 256u * ks, 128, 512);
                        tc::mma_bf16(tmem, ah, b, id_v, (kc > 0 || ks > 0) ? 1u : 0u);
                        tc::mma_bf16(tmem, al, b, id_v, 1u);
                    }
                    tc::commit(mbar);
                }
                ok = __syncthreads_and(tc::mbar_wait(mbar, phase, kMaxTries) ? 1 : 0) != 0;
                phase ^= 1u;
            }
            if (!ok) break;
            tc::fence_after();
            float hh = 0.f;
            for (int cb = 0; cb < n; cb += 32) {
                float v[32];
                tc::tmem_ld32(tmem + lane_off + (uint32_t)cb, v);
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const float2 ge = gs[(size_t)(cb + j) * TP + tid];
                    hh = fmaf(ge.x * ge.x + ge.y * ge.y, v[j], hh);
                }
            }
            hh *= fc.w4;
            if (valid && A.h_out) A.h_out[(size_t)fw * G.npix + px] = hh;
            acc_h += hh;
            tc::fence_before();
            __syncthreads();
        }
        if (ok && valid) {
            if (A.gsum) A.gsum[px] = acc_g;
            if (A.hsum) A.hsum[px] = acc_h;
        }
    }
    if (!ok) {
        // a wait ran out: report it, give the tensor core a bounded last chance to drain, then free TMEM
        if (tid == 0) atomicAdd(A.counters + CNT_TC_TIMEOUT, 1u);
        tc::mbar_wait(mbar, phase ^ 1u, kMaxTries);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, A.tmem_cols);
}

}  // namespace

bool tc_adjoint_supported(int n_elem) { return n_elem >= 32 && n_elem <= 256 && n_elem % 32 == 0; }

size_t tc_b_images_bytes(int n_elem) {
    const size_t n = (size_t)n_elem;
    return (2 * n) * (2 * n) * 2 * 2 + n * n * 2;   // bu (hi + lo) + bw, bf16
}

cudaError_t launch_prep_b(int n, const float2* R, const uint8_t* W, void* img, cudaStream_t s) {
    __nv_bfloat16* bu = (__nv_bfloat16*)img;
    __nv_bfloat16* bw = bu + (size_t)(2 * n) * (2 * n) * 2;
    k_prep_b<<<256, 256, 0, s>>>(n, R, W, bu, bw);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_tc(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F,
                              const void* images, float2* gscr, int n_ctas, float2* g_out, float* h_out, float* gsum,
                              float* hsum, uint32_t* counters, cudaStream_t s) {
    const int n = G.n_elem;
    if (!tc_adjoint_supported(n)) return cudaErrorInvalidValue;
    TcArgs A;
    A.G = G;
    A.F = F;
    A.tables = tables;
    A.c = c;
    A.bu = (const __nv_bfloat16*)images;
    A.bu_stride = tc_b_images_bytes(n) / 2;
    A.bw = A.bu + (size_t)(2 * n) * (2 * n) * 2;
    A.bw_stride = A.bu_stride;
    A.gscr = gscr;
    A.g_out = g_out;
    A.h_out = h_out;
    A.gsum = gsum;
    A.hsum = hsum;
    A.counters = counters;
    A.n_tiles = (G.npix + TP - 1) / TP;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * n)) cols <<= 1;
    A.tmem_cols = cols;
    // more than half of the SM's shared memory: one CTA (one TMEM owner) per SM
    const int sm = 120 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    const int grid = n_ctas < A.n_tiles ? n_ctas : A.n_tiles;
    k_adjoint_tc<<<grid, NTHR, sm, s>>>(A);
    return cudaGetLastError();
}
