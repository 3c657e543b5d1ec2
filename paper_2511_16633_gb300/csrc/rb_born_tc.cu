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
#include <cuda.h>

#include "rb_internal.cuh"
#include "rb_tc.cuh"

namespace {

constexpr int TP = RB_TP;               // pixels per tile = MMA M
constexpr uint32_t kMaxTries = 1u << 22; // mbarrier polls before giving up (each poll suspends briefly)

// ---------------------------------------------------------------------------
// B operand images for one frequency, in K slices of 16 (one pipeline stage each)
// in the core-matrix layout of rb_tc.cuh (tile16_offset).
//   bu: [ks = 2n/16][hi|lo][2n rows x 16]   (2n rows = e', K = 2n)
//   bw: [ks = n/32][n rows x 32]            (W, exact; K = 32 slices, chunk_offset)
// ---------------------------------------------------------------------------
__global__ void k_prep_b(int n, const float2* __restrict__ R, const uint8_t* __restrict__ W,
                         __nv_bfloat16* __restrict__ bu, __nv_bfloat16* __restrict__ bw) {
    const int n2 = 2 * n;
    const size_t img_u = (size_t)n2 * 16;  // bf16 per hi or lo image of one slice
    const long long total_u = (long long)n2 * n2;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total_u;
         j += (long long)gridDim.x * blockDim.x) {
        const int ep = (int)(j / n2), kp = (int)(j % n2);
        const int r = kp >> 1, part = kp & 1;
        // rows e' in N-blocks of nb columns (the adjoint's MMA width), each holding the
        // Re U rows then the Im U rows of nb / 2 consecutive elements; a pass of the
        // adjoint takes ne2 = 2 min(n, 256) rows in one or two N-blocks
        const int ne2 = n2 < 512 ? n2 : 512;
        const int nb = ne2 > 256 ? ne2 / 2 : ne2, eb = nb / 2;
        const int blk = ep / nb, w = ep % nb;
        const int e = blk * eb + w % eb, im = w / eb;
        float2 s = make_float2(0.f, 0.f);
        if (W[(size_t)e * n + r]) s = R[(size_t)e * n + r];
        float v;
        if (im == 0) v = part == 0 ? s.x : -s.y;
        else v = part == 0 ? s.y : s.x;
        __nv_bfloat16 hi, lo;
        tc::split_bf16(v, hi, lo);
        const int ks = kp >> 4, kk = kp & 15;
        const size_t base = (size_t)ks * 2 * img_u;
        const uint32_t off = tc::tile16_offset((uint32_t)ep, (uint32_t)kk) / 2;
        bu[base + off] = hi;
        bu[base + img_u + off] = lo;
    }
    const long long total_w = (long long)n * n;
    const size_t img_w = (size_t)n * 32;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total_w;
         j += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(j / n), r = (int)(j % n);
        const int ks = r >> 5, kk = r & 31;
        bw[(size_t)ks * img_w + tc::chunk_offset((uint32_t)e, (uint32_t)kk) / 2] =
            __float2bfloat16_rn(W[(size_t)e * n + r] ? 1.f : 0.f);
    }
}

struct TcArgs {
    GeoDev G;
    FreqSet F;
    const __nv_bfloat16* aimg; // [n_freq][tiles][hi|lo][2n / 8 rows][1024] A image (layout: aimg_put4)
    size_t aimg_stride;        // bf16 elements per frequency
    const __nv_bfloat16* bu;   // [n_freq][image]
    const __nv_bfloat16* bw;   // [n_freq][image]
    size_t bu_stride, bw_stride;  // bf16 elements per frequency
    float2* gscr;              // [gridDim.x][n][TP] exact G per CTA
    __nv_bfloat16* vimg;       // [gridDim.x][n / 32][hi|lo][TP x 32] |G|^2 A slices of the Hessian contraction
    float2* g_out;             // [n_freq][npix] or null
    float* h_out;              // [n_freq][npix] or null
    float* gsum;               // [npix] or null (sum over w of Re g)
    float* hsum;               // [npix] or null
    float2* fpart;             // [n_freq][npix] (Re g, H) of each frequency for k_adjoint_sums, or null
    uint32_t* counters;
    int n_tiles;
    uint32_t tmem_cols;
    int n_e, npass;            // elements per pass (N of the MMAs: 2 n_e and n_e), passes = n / n_e
    int want_h;                // the Hessian contraction is wanted (h_out or hsum set)
};

}  // namespace

namespace {

// Pipeline shapes of the tensor-core kernels.
constexpr int NPROD = 512;                   // adjoint producer threads: four per pixel row
constexpr int NTHR_A = NPROD + 64;           // + MMA warp + B-loader warp
constexpr int NPROD_F = 256;                 // forward producer threads: two per A row
constexpr int NTHR_F = NPROD_F + 64;
constexpr int NST = 5;                       // pipeline stages
constexpr uint32_t ST_BYTES = 40u * 1024u;   // A hi (4 KB) + A lo (4 KB) + B (<= 32 KB)
constexpr uint32_t ST_ALO = 4096u, ST_B = 8192u;
// V slices of the adjoint (K = 32): A hi (8 KB) + A lo (8 KB) + W (n rows x 32, <= 16 KB)
constexpr uint32_t ST_VALO = 8192u, ST_VB = 16384u;

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// |G|^2 of elements e .. e + 7 (e a multiple of 8) at pixel p, hi and lo planes, from the
// tile's V A slices (written by consume_u; K = 32 slices in the chunk_offset layout, so
// the 8 values of a plane are 16 contiguous bytes): half the bytes of reading G back.
__device__ __forceinline__ void g2_load(const __nv_bfloat16* vimg, int e, uint32_t p, uint4 (&q)[2]) {
    const __nv_bfloat16* vs = vimg + (size_t)(e >> 5) * (2 * TP * 32);
    const uint32_t vo = tc::chunk_offset(p, (uint32_t)(e & 31)) / 2;
    q[0] = *(const uint4*)(vs + vo);
    q[1] = *(const uint4*)(vs + TP * 32 + vo);
}

// hh += sum_i |G_i|^2 V_i over a chunk of 8 elements: V from TMEM (8 columns at taddr),
// |G|^2 = hi + lo (the values the V MMAs used).
__device__ __forceinline__ void h_chunk(uint32_t taddr, const uint4 (&q)[2], float& hh) {
    float v[8];
    tc::tmem_ld8(taddr, v);
    const uint32_t wh[4] = {q[0].x, q[0].y, q[0].z, q[0].w}, wl[4] = {q[1].x, q[1].y, q[1].z, q[1].w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float g0 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(wh[i] & 0xffffu))) +
                         __bfloat162float(__ushort_as_bfloat16((unsigned short)(wl[i] & 0xffffu)));
        const float g1 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(wh[i] >> 16))) +
                         __bfloat162float(__ushort_as_bfloat16((unsigned short)(wl[i] >> 16)));
        hh = fmaf(g0, v[2 * i], hh);
        hh = fmaf(g1, v[2 * i + 1], hh);
    }
}

// Producer work of one U slice (8 elements, K' = 16) for thread (p, h), h < 4: the
// A slice in shared memory (two rows of the A image, layout of aimg_put4) holds, at
// K' positions 4h .. 4h + 3 of row p, the bf16
// hi / lo parts of (Re G, -Im G) of elements r0 + 2h + j (j < 2).  Their sums give
// G to ~2^-17 relative for the epilogue (gs), and |G|^2 (hi / lo) goes to the V
// slice r0 / 16 of this CTA.
__device__ __forceinline__ void consume_u(int r0, uint32_t p, uint32_t h, const unsigned char* a_hi,
                                          const unsigned char* a_lo, float2* gs, __nv_bfloat16* vimg, bool want_h) {
    // A slice = two image rows (K cores) of 2 KB: K core h / 2, pixel core p / 8, row p % 8
    const uint32_t off = (h >> 1) * 2048u + (p >> 3) * 128u + (p & 7u) * 16u + 8u * (h & 1u);
    const uint2 wh = *(const uint2*)(a_hi + off), wl = *(const uint2*)(a_lo + off);
    const uint32_t hw[2] = {wh.x, wh.y}, lw[2] = {wl.x, wl.y};
    __nv_bfloat16 vh[2], vl[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float re = __bfloat162float(__ushort_as_bfloat16((unsigned short)(hw[j] & 0xffffu))) +
                         __bfloat162float(__ushort_as_bfloat16((unsigned short)(lw[j] & 0xffffu)));
        const float mim = __bfloat162float(__ushort_as_bfloat16((unsigned short)(hw[j] >> 16))) +
                          __bfloat162float(__ushort_as_bfloat16((unsigned short)(lw[j] >> 16)));
        gs[(size_t)(r0 + 2 * (int)h + j) * TP + p] = make_float2(re, -mim);
        tc::split_bf16(re * re + mim * mim, vh[j], vl[j]);
    }
    if (!want_h) return;
    __nv_bfloat16* vs = vimg + (size_t)(r0 >> 5) * (2 * TP * 32);
    const uint32_t voff = tc::chunk_offset(p, (uint32_t)(r0 & 31) + 2u * h) / 2;
    *(uint32_t*)(vs + voff) = pack2(vh[0], vh[1]);
    *(uint32_t*)(vs + TP * 32 + voff) = pack2(vl[0], vl[1]);
}

// ---------------------------------------------------------------------------
// Operand image of one frequency set (layout: aimg_put4 in rb_internal.cuh) from the
// caller's tables, for the single-operator entry points (the update writes it from its
// resolve pass: k_resolve_images, rb_trace.cu).  The synthesis record of each entry is
// formed in registers from its table record, c at the pixel and the distance to the
// element.  The adjoint reads the image K-major (a K = 16 slice is two rows: one 4 KB
// bulk copy per plane), the forward MN-major (a 16-pixel slice of every row is one 2-D
// TMA box).  CTA (tile, element block of 16): thread (p, half) synthesises elements
// 16 eb + 8 half + k (k < 8) at pixel p for every frequency and writes rows
// 4 eb + 2 half + {0, 1} of the pixel's core row (coalesced: 128 threads, 2 KB).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tables_images(GeoDev G, const rb_cell* __restrict__ tables,
                                                       const float* __restrict__ c, FreqSet F,
                                                       __nv_bfloat16* __restrict__ aimg, size_t a_stride) {
    const int n = G.n_elem, rcn = 2 * n / 8;
    const int neb = n / 16;
    const int tile = (int)blockIdx.x / neb, eb = (int)blockIdx.x % neb;
    const int tid = threadIdx.x, p = tid & (TP - 1), half = tid >> 7;
    const int px = tile * TP + p;
    const int e0 = 16 * eb + 8 * half;
    float4 sr[8];
    if (px < G.npix) {
        const float c_px = __ldg(c + px);
        const int ix = px % G.nx, iy = px / G.nx;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            DF ex, ey;
            elem_pos(G, e0 + k, ex, ey);
            sr[k] = synth_record(tables[(size_t)(e0 + k) * G.npix + px], c_px, pixel_elem_dist(G, ix, iy, ex, ey),
                                 G.inv_cref, G.inv_cref_lo, G.j_floor);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) sr[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int fw = 0; fw < F.n; ++fw) {
        const FreqC& fc = F.f[fw];
        __nv_bfloat16* plane = aimg + (size_t)fw * a_stride + (size_t)tile * 2 * rcn * 1024;
#pragma unroll
        for (int kg = 0; kg < 2; ++kg) {
            float2 g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q] = green_srec(sr[4 * kg + q], fc);
            aimg_put4(plane, rcn, 4 * eb + 2 * half + kg, p, g);
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint kernel: warp-specialised, NST-stage pipeline of K = 16 slices.
//   warps 0..15 producers: from each U slice's A (in shared memory, items of 8
//               pixels x 4 K quarters per warp) they keep G for the epilogue (gs)
//               and write the |G|^2 A slices of V; then the epilogues (TMEM ->
//               registers; thread = pixel p = tid % 128, the TMEM lane, and quarter
//               h = tid / 128 of the elements);
//   warp 16     MMA issuer (lane 0): waits for a stage, issues its MMAs and
//               commits their completion to the stage's "empty" barrier;
//   warp 17     loader (lane 0): bulk-copies A and B of each slice (U: the A image
//               and S; V: the |G|^2 slices and W) into a stage as soon as the
//               stage's previous contents have been used.
// Per (tile, frequency, pass over the elements) the slice sequence is U (2n / 16
// slices of K = 16) then, when the Hessian diagonal is wanted, V (n / 32 slices of
// K = 32); a pass covers 256 elements of e (all of them up to 256 elements), the
// contractions always run over all of r.
// Barriers: full[s] (bulk-copy bytes), empty[s] (the MMAs that read stage s done,
// plus 16 producer-warp arrivals: A read), acc_full (last MMA of a phase done),
// acc_empty (16 producer-warp arrivals: the epilogue has read the accumulator),
// vready (16 producer-warp arrivals: the |G|^2 slices of this tile are written),
// drain (MMA completion on the error path).  Every wait is bounded; a timeout
// raises a shared flag that ends all loops.
// ---------------------------------------------------------------------------
// MULTI: more than one pass over the elements (rings above 256 elements, passes of 256);
// the one-pass kernel is compiled without the pass bookkeeping.
template <bool MULTI>
__global__ void __launch_bounds__(NTHR_A, 1) k_adjoint_tc(TcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_full[NST], s_empty[NST], s_acc_full, s_acc_empty, s_acc_low, s_vready, s_drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_err;
    __shared__ float s_red[3][3][TP];             // partial sums of quarters 1..3: Re g, Im g, H
    const GeoDev& G = A.G;
    const int n = G.n_elem, n2 = 2 * n;
    // the elements e of U and V are taken in passes of ne (the accumulators of one pass
    // fit TMEM); the contractions run over all r in every pass
    const int ne = A.n_e, ne2 = 2 * ne;
    const int npass = MULTI ? A.npass : 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // U slices, then (when the Hessian diagonal is wanted) V slices
    const bool want_h = A.want_h != 0;
    const int nU = n2 / 16, nV = want_h ? n / 32 : 0, per = nU + nV;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            tc::mbar_init(tc::smem_u32(&s_full[s]), 1);
            tc::mbar_init(tc::smem_u32(&s_empty[s]), 1 + NPROD / 32);
        }
        tc::mbar_init(tc::smem_u32(&s_acc_full), 1);
        tc::mbar_init(tc::smem_u32(&s_acc_empty), NPROD / 32);
        tc::mbar_init(tc::smem_u32(&s_acc_low), NPROD / 32);
        tc::mbar_init(tc::smem_u32(&s_vready), NPROD / 32);
        tc::mbar_init(tc::smem_u32(&s_drain), 1);
        s_err = 0;
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), A.tmem_cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    __nv_bfloat16* vimg = A.vimg + (size_t)blockIdx.x * (size_t)(n / 32) * (2 * TP * 32);
    const int n_items = A.n_tiles * A.F.n;
    const int my_items = (int)blockIdx.x < n_items ? (n_items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // slices of this CTA (a few thousand: 32-bit counters, stage and phase advanced
    // incrementally, no divisions in the loops)
    const int total = my_items * npass * per;
    const size_t img_u = (size_t)n2 * 16, img_w = (size_t)n * 32;  // bf16 per hi (or lo) / W image slice
    auto stage = [&](int s) { return smem + (size_t)s * ST_BYTES; };

    if (warp == NPROD / 32 + 1) {
        // ------------------------------ loader ------------------------------
        if (lane == 0) {
            int ql = 0, s = 0, j = 0, pass = 0, item = blockIdx.x;
            int tile = item / A.F.n, fw = item - tile * A.F.n;
            uint32_t ph = 0, vrp = 0;
            bool err = false;
            // the operand image streams through L2 once per launch: first out, so that it does
            // not push the CTAs' G and |G|^2 scratch (rewritten every tile) out to DRAM
            uint64_t stream_pol;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_pol));
            for (; ql < total; ++ql) {
                // stage s = ql % NST with phase ph = (ql / NST) & 1; slice j of frequency fw of tile
                if (ql >= NST && !tc::mbar_wait(tc::smem_u32(&s_empty[s]), ph ^ 1u, kMaxTries)) {
                    err = true;
                    break;
                }
                if (s_err) break;
                const uint32_t mb = tc::smem_u32(&s_full[s]);
                if (j < nU) {
                    const uint32_t abytes = TP * 16 * 2, bbytes = (uint32_t)(ne2 * 64);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(2u * abytes + bbytes)
                                 : "memory");
                    // image rows 2j, 2j + 1 of the hi plane, then of the lo plane
                    const __nv_bfloat16* asrc =
                        A.aimg + (size_t)fw * A.aimg_stride + ((size_t)tile * 2 * (n2 / 8) + 2 * j) * 1024;
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                                 " [%0], [%1], %2, [%3], %4;"
                                 ::"r"(tc::smem_u32(stage(s))), "l"(asrc), "r"(abytes), "r"(mb), "l"(stream_pol)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                                 " [%0], [%1], %2, [%3], %4;"
                                 ::"r"(tc::smem_u32(stage(s) + ST_ALO)), "l"(asrc + (size_t)(n2 / 8) * 1024), "r"(abytes),
                                 "r"(mb), "l"(stream_pol)
                                 : "memory");
                    // B: rows e' of this pass (contiguous in each plane), hi then lo; with one
                    // pass the two planes are adjacent and go in one copy
                    const __nv_bfloat16* bsrc = A.bu + (size_t)fw * A.bu_stride + (size_t)j * 2 * img_u + (size_t)pass * ne2 * 16;
                    if (!MULTI) {
                        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                     ::"r"(tc::smem_u32(stage(s) + ST_B)), "l"(bsrc), "r"(bbytes), "r"(mb)
                                     : "memory");
                    } else {
                        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                     ::"r"(tc::smem_u32(stage(s) + ST_B)), "l"(bsrc), "r"(bbytes / 2), "r"(mb)
                                     : "memory");
                        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                     ::"r"(tc::smem_u32(stage(s) + ST_B + bbytes / 2)), "l"(bsrc + img_u), "r"(bbytes / 2),
                                     "r"(mb)
                                     : "memory");
                    }
                } else {
                    if (j == nU) {
                        // this (tile, frequency)'s |G|^2 slices are written by the producers
                        if (!tc::mbar_wait(tc::smem_u32(&s_vready), vrp & 1u, kMaxTries)) {
                            err = true;
                            break;
                        }
                        ++vrp;
                    }
                    const uint32_t wbytes = (uint32_t)(ne * 64), abytes = 2u * TP * 32 * 2;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(wbytes + abytes)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(tc::smem_u32(stage(s) + ST_VB)),
                                 "l"(A.bw + (size_t)fw * A.bw_stride + (size_t)(j - nU) * img_w + (size_t)pass * ne * 32),
                                 "r"(wbytes), "r"(mb)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(tc::smem_u32(stage(s))), "l"(vimg + (size_t)(j - nU) * (2 * TP * 32)), "r"(abytes),
                                 "r"(mb)
                                 : "memory");
                }
                if (++s == NST) { s = 0; ph ^= 1u; }
                if (++j == per) {
                    j = 0;
                    if (++pass == npass) {
                        pass = 0;
                        item += gridDim.x;
                        tile = item / A.F.n;
                        fw = item - tile * A.F.n;
                    }
                }
            }
            if (err || s_err) {
                s_err = 1;
                // bounded waits for the last copies issued (at most one per stage)
                for (int x = (ql > NST ? ql - NST : 0); x < ql; ++x)
                    tc::mbar_wait(tc::smem_u32(&s_full[x % NST]), (uint32_t)(x / NST) & 1u, kMaxTries);
            }
        }
        __syncwarp();
    } else if (warp == NPROD / 32) {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            const int nbk = ne2 > 256 ? 2 : 1;
            const int nb_u = ne2 / nbk;
            const uint32_t id_u = tc::idesc_bf16_f32(128, (uint32_t)nb_u);
            const uint32_t id_v = tc::idesc_bf16_f32(128, (uint32_t)ne);
            int s = 0, j = 0;
            uint32_t acce = 0, accl = 0, ph = 0;
            bool err = false, issued = false;
            for (int q = 0; q < total && !err; ++q) {
                if (j == nU) {
                    // V overwrites the columns of the first N-block of U: its part of the U
                    // epilogue must be done (the rest of it overlaps the V MMAs)
                    if (!tc::mbar_wait(tc::smem_u32(&s_acc_low), accl & 1u, kMaxTries)) { err = true; break; }
                    ++accl;
                } else if (j == 0 && q > 0) {
                    // a new U phase: the V epilogue must have read the accumulator
                    if (!tc::mbar_wait(tc::smem_u32(&s_acc_empty), acce & 1u, kMaxTries)) { err = true; break; }
                    ++acce;
                }
                if (!tc::mbar_wait(tc::smem_u32(&s_full[s]), ph, kMaxTries)) { err = true; break; }
                if (s_err) { err = true; break; }
                tc::fence_after();
                const uint32_t sa = tc::smem_u32(stage(s)), sal = sa + ST_ALO, sb = sa + ST_B;
                // U: A K-major in the image's arrangement: K cores 2048 B apart (LBO), 8-pixel
                // cores 128 B apart (SBO)
                const uint64_t dah = tc::sdesc(sa, 2048, 128), dal = tc::sdesc(sal, 2048, 128);
                if (j < nU) {
                    const uint32_t acc = j > 0 ? 1u : 0u;
                    for (int nb = 0; nb < nbk; ++nb) {
                        const uint32_t boff = (uint32_t)(nb * nb_u / 8) * 256u;
                        const uint64_t dbh = tc::sdesc(sb + boff, 128, 256);
                        const uint64_t dbl = tc::sdesc(sb + (uint32_t)(ne2 * 32) + boff, 128, 256);
                        const uint32_t d = tmem + (uint32_t)(nb * nb_u);
                        tc::mma_bf16(d, dah, dbh, id_u, acc);
                        tc::mma_bf16(d, dah, dbl, id_u, 1u);
                        tc::mma_bf16(d, dal, dbh, id_u, 1u);
                    }
                } else {
                    // K = 32 slice in the chunk_offset layout (SBO = 512): two K = 16 steps
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        const uint64_t vah = tc::sdesc(sa + 256u * kh, 128, 512);
                        const uint64_t val = tc::sdesc(sa + ST_VALO + 256u * kh, 128, 512);
                        const uint64_t vb = tc::sdesc(sa + ST_VB + 256u * kh, 128, 512);
                        tc::mma_bf16(tmem, vah, vb, id_v, (j > nU || kh > 0) ? 1u : 0u);
                        tc::mma_bf16(tmem, val, vb, id_v, 1u);
                    }
                }
                issued = true;
                tc::commit(tc::smem_u32(&s_empty[s]));
                if (j == nU - 1 || j == per - 1) tc::commit(tc::smem_u32(&s_acc_full));
                if (++s == NST) { s = 0; ph ^= 1u; }
                if (++j == per) j = 0;
            }
            if (err) {
                s_err = 1;
                atomicAdd(A.counters + CNT_TC_TIMEOUT, 1u);
                // bounded wait for the MMAs still in flight
                if (issued) {
                    tc::commit(tc::smem_u32(&s_drain));
                    tc::mbar_wait(tc::smem_u32(&s_drain), 0u, kMaxTries);
                }
            }
        }
        __syncwarp();
    } else {
        // -------------------------------- producers --------------------------------
        const uint32_t p = (uint32_t)(tid & (TP - 1)), h = (uint32_t)(tid / TP);
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        // the U slices' (pixel, quarter) items go 8 pixels x 4 quarters to a warp: the A reads
        // then fall on distinct shared-memory banks and the |G|^2 stores on 128 contiguous
        // bytes (the epilogues keep p = the TMEM lane)
        const uint32_t cp = (uint32_t)((lane & 7) + 8 * warp), ch = (uint32_t)(lane >> 3);
        float2* gs = A.gscr + (size_t)blockIdx.x * n * TP;
        bool err = false;
        int qs = 0;                // stage of the next slice
        uint32_t qph = 0;          // its phase
        uint32_t accf = 0;
        // one slice: wait for its stage to be filled, use it, release it
        auto slice = [&](auto&& consume) {
            const int s = qs;
            if (!err) err = !tc::mbar_wait(tc::smem_u32(&s_full[s]), qph, kMaxTries);
            err = __any_sync(0xffffffffu, err || s_err != 0);
            if (!err) consume(stage(s), stage(s) + ST_ALO);
            __syncwarp();
            if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_empty[s]));
            if (++qs == NST) { qs = 0; qph ^= 1u; }
        };
        // wait for the accumulator of the phase just issued (warp-uniform result)
        auto acc_wait = [&]() {
            if (!err) err = !tc::mbar_wait(tc::smem_u32(&s_acc_full), accf & 1u, kMaxTries);
            ++accf;
            err = __any_sync(0xffffffffu, err);
            tc::fence_after();
        };
        auto acc_release = [&]() {
            tc::fence_before();
            __syncwarp();
            if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_acc_empty));
        };
        // items (tile, frequency), item = tile F.n + fw, dealt to the CTAs in turn
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int tile = item / A.F.n, fw = item - (item / A.F.n) * A.F.n;
            const int px = tile * TP + (int)p;
            const bool valid = px < G.npix;
            {
                const FreqC fc = A.F.f[fw];
                float fg_r = 0.f, fg_i = 0.f, fh = 0.f;   // this frequency's g and H, summed over the passes
                for (int pass = 0; pass < npass; ++pass) {
                const int eb0 = pass * ne;                 // first element of this pass
                // ---- U slices: exact-enough G for the epilogue and the |G|^2 slices ----
                for (int j = 0; j < nU; ++j)
                    slice([&](const unsigned char* ahi, const unsigned char* alo) {
                        consume_u(j * 8, cp, ch, ahi, alo, gs, vimg, want_h);
                    });
                // the |G|^2 slices (read next by the bulk copies of the loader) are complete
                if (want_h) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_vready));
                }
                // gs (G of the tile) is complete
                err = tc::named_or(1, NPROD, err);
                if (err) break;
                // ---- U epilogue: element chunks of 8, e0 = 32 b + 8 c for blocks b = h, h + 4, ...
                // and c < 4 (in increasing e); element e's Re U is in column nbu (e / ebu) + e % ebu
                // and its Im U ebu columns further (N-blocks of nbu columns, ebu = nbu / 2
                // elements each); G of the next chunk is loaded while the current one is used,
                // the first before the accumulator wait ----
                const int nch = 4 * ((ne / 32 - (int)h + 3) / 4);
                const int nbu = ne2 > 256 ? ne2 / 2 : ne2, ebu = nbu / 2;
                auto ce0 = [&](int k) { return 32 * ((int)h + 4 * (k >> 2)) + 8 * (k & 3); };
                auto recol = [&](int e) { return (e / ebu) * nbu + e % ebu; };
                auto gload = [&](int k, float2 (&g)[8]) {
                    const int e0 = ce0(k);
#pragma unroll
                    for (int i = 0; i < 8; ++i) g[i] = gs[(size_t)(eb0 + e0 + i) * TP + p];
                };
                auto gchunk = [&](int k, const float2 (&g)[8], float& ar, float& ai) {
                    const int e0 = ce0(k);
                    float vr[8], vi[8];
                    tc::tmem_ld8(tmem + lane_off + (uint32_t)recol(e0), vr);
                    tc::tmem_ld8(tmem + lane_off + (uint32_t)(recol(e0) + ebu), vi);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        ar = fmaf(g[i].x, vr[i], fmaf(g[i].y, vi[i], ar));
                        ai = fmaf(g[i].x, vi[i], fmaf(-g[i].y, vr[i], ai));
                    }
                };
                // the V MMAs write columns [0, n), inside the first N-block: released once this
                // warp has read its chunks of elements < ebu
                bool low = false;
                auto release_low = [&]() {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_acc_low));
                    low = true;
                };
                float2 ga[8], gb[8];
                if (nch > 0) gload(0, ga);
                acc_wait();
                float gr = 0.f, gi = 0.f;
                if (!err) {
                    for (int k = 0; k < nch; k += 2) {
                        if (!low && ce0(k) >= ebu) release_low();
                        gload(k + 1, gb);
                        gchunk(k, ga, gr, gi);
                        if (k + 2 < nch) gload(k + 2, ga);
                        gchunk(k + 1, gb, gr, gi);
                    }
                }
                if (!low) release_low();
                if (h > 0) {
                    s_red[0][h - 1][p] = gr;
                    s_red[1][h - 1][p] = gi;
                }
                err = tc::named_or(1, NPROD, err);
                if (err) break;
                if (h == 0) {
                    fg_r += (gr + s_red[0][0][p] + s_red[0][1][p] + s_red[0][2][p]) * fc.w2;
                    fg_i += (gi + s_red[1][0][p] + s_red[1][1][p] + s_red[1][2][p]) * fc.w2;
                }
                if (!want_h) {
                    // no V phase: the accumulator is free for the next U phase
                    acc_release();
                    continue;
                }
                // ---- V slices: A and B come by bulk copy; the producers only pass the
                // stage barriers, which keeps every stage's phases in step with its uses ----
                for (int j = 0; j < nV; ++j) slice([&](const unsigned char*, const unsigned char*) {});
                // ---- V epilogue (same chunks, |G|^2 against V in columns e) ----
                uint4 qa[2], qb[2];
                if (nch > 0) g2_load(vimg, eb0 + ce0(0), p, qa);
                acc_wait();
                float hh = 0.f;
                if (!err) {
                    for (int k = 0; k < nch; k += 2) {
                        g2_load(vimg, eb0 + ce0(k + 1), p, qb);
                        h_chunk(tmem + lane_off + (uint32_t)ce0(k), qa, hh);
                        if (k + 2 < nch) g2_load(vimg, eb0 + ce0(k + 2), p, qa);
                        h_chunk(tmem + lane_off + (uint32_t)ce0(k + 1), qb, hh);
                    }
                }
                acc_release();
                if (h > 0) s_red[2][h - 1][p] = hh;
                err = tc::named_or(1, NPROD, err);
                if (err) break;
                if (h == 0) fh += (hh + s_red[2][0][p] + s_red[2][1][p] + s_red[2][2][p]) * fc.w4;
                }   // passes
                if (err) break;
                if (h == 0 && valid) {
                    if (A.g_out) A.g_out[(size_t)fw * G.npix + px] = make_float2(fg_r, fg_i);
                    if (A.h_out) A.h_out[(size_t)fw * G.npix + px] = fh;
                    // this frequency's Re g and H for the sums over the set (k_adjoint_sums)
                    if (A.fpart) A.fpart[(size_t)fw * G.npix + px] = make_float2(fg_r, fh);
                }
            }
            if (err) break;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, A.tmem_cols);
}
// ---------------------------------------------------------------------------
// The same adjoint on CTA pairs (a cluster of two CTAs, cta_group::2 MMAs of M = 256).
// The pair takes two 128-pixel tiles at a time, one per CTA (a pair with one tile left
// takes the last tile twice and keeps one result), and each CTA stages only its own
// half of every operand: its tile's A slices and half the rows of each N-block of S
// (and of W).  The MMA over both CTAs' shared memory then reads half the S bytes per
// CTA that the single-CTA kernel reads, and the stages (A 8 KB + S half 16 KB) are
// 24 KB instead of 40, so eight of them fit.  Each CTA's TMEM holds its own tile's U
// and V (128 lanes), so the producers and epilogues are those of the single-CTA
// kernel.  Roles as there, plus:
//   rank 0, warp 16: MMA issuer for the pair: waits for its own stage and for the
//               peer's ("pfull", arrived on from the peer), issues the pair MMAs and
//               commits them to the "empty" (and accumulator) barriers of both CTAs;
//   rank 1, warp 16: relay: when a stage of its CTA is filled, arrives on the
//               issuer's pfull for it;
//   the accumulator barriers the issuer waits for (acc_empty, acc_low) take the
//   arrivals of both CTAs' producer warps.
// Every wait is bounded; both CTAs meet at a cluster barrier before they free TMEM
// and exit, so no CTA leaves while its peer may still touch its shared memory.
// ---------------------------------------------------------------------------
constexpr int NST2 = 8;
constexpr uint32_t ST2_BYTES = 24u * 1024u;
// U stage: A hi (4 KB), A lo (4 KB), then this CTA's S rows of every N-block (hi for each
// N-block, then lo); V stage: |G|^2 hi (8 KB), lo (8 KB), this CTA's W rows (<= 8 KB)
constexpr uint32_t ST2_ALO = 4096u, ST2_B = 8192u, ST2_VALO = 8192u, ST2_VB = 16384u;

template <bool MULTI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHR_A, 1) k_adjoint_tc2(TcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_full[NST2], s_pfull[NST2], s_empty[NST2], s_acc_full, s_acc_empty, s_acc_low, s_vready, s_drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_err;
    __shared__ float s_red[3][3][TP];             // partial sums of quarters 1..3: Re g, Im g, H
    const GeoDev& G = A.G;
    const int n = G.n_elem, n2 = 2 * n;
    const int ne = A.n_e, ne2 = 2 * ne;
    const int npass = MULTI ? A.npass : 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = tc::cluster_ctarank();   // 0 issues the pair's MMAs
    const bool want_h = A.want_h != 0;
    const int nU = n2 / 16, nV = want_h ? n / 32 : 0, per = nU + nV;
    // N-blocks of U (as in the single-CTA kernel) and this CTA's half of each
    const int nbk = ne2 > 256 ? 2 : 1, nb_u = ne2 / nbk, hrow = nb_u / 2;
    const uint32_t hb = (uint32_t)hrow * 32u;    // bytes of one plane of one N-block half
    const int wrow = ne / 2;                     // this CTA's W rows
    if (tid == 0) {
        for (int s = 0; s < NST2; ++s) {
            tc::mbar_init(tc::smem_u32(&s_full[s]), 1);
            tc::mbar_init(tc::smem_u32(&s_pfull[s]), 1);
            tc::mbar_init(tc::smem_u32(&s_empty[s]), 1 + NPROD / 32);
        }
        tc::mbar_init(tc::smem_u32(&s_acc_full), 1);
        tc::mbar_init(tc::smem_u32(&s_acc_empty), 2 * NPROD / 32);
        tc::mbar_init(tc::smem_u32(&s_acc_low), 2 * NPROD / 32);
        tc::mbar_init(tc::smem_u32(&s_vready), NPROD / 32);
        tc::mbar_init(tc::smem_u32(&s_drain), 1);
        s_err = 0;
    }
    if (warp == 0) tc::tmem_alloc_pair(tc::smem_u32(&s_tmem), A.tmem_cols);
    tc::fence_before();
    tc::cluster_sync();   // both CTAs' barriers initialised before any cross-CTA arrival
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    __nv_bfloat16* vimg = A.vimg + (size_t)blockIdx.x * (size_t)(n / 32) * (2 * TP * 32);
    const int n_pairs = (A.n_tiles + 1) / 2, q0 = (int)blockIdx.x >> 1, nq = (int)gridDim.x >> 1;
    const int my_items = q0 < n_pairs ? (n_pairs - 1 - q0) / nq + 1 : 0;
    const int total = my_items * A.F.n * npass * per;
    const size_t img_u = (size_t)n2 * 16, img_w = (size_t)n * 32;
    auto stage = [&](int s) { return smem + (size_t)s * ST2_BYTES; };
    // this CTA's tile of pair item q (the last tile again when the pair has only one)
    auto tile_of = [&](int q) {
        const int t = 2 * q + (int)rank;
        return t < A.n_tiles ? t : A.n_tiles - 1;
    };

    if (warp == NPROD / 32 + 1) {
        // ------------------------------ loader (both CTAs) ------------------------------
        if (lane == 0) {
            int ql = 0, s = 0, j = 0, fw = 0, pass = 0, q = q0;
            uint32_t ph = 0, vrp = 0;
            bool err = false;
            uint64_t stream_pol;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_pol));
            for (; ql < total; ++ql) {
                if (ql >= NST2 && !tc::mbar_wait(tc::smem_u32(&s_empty[s]), ph ^ 1u, kMaxTries)) {
                    err = true;
                    break;
                }
                if (s_err) break;
                const uint32_t mb = tc::smem_u32(&s_full[s]);
                const int tile = tile_of(q);
                if (j < nU) {
                    const uint32_t abytes = TP * 16 * 2;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                                 "r"(2u * abytes + 2u * (uint32_t)nbk * hb)
                                 : "memory");
                    const __nv_bfloat16* asrc =
                        A.aimg + (size_t)fw * A.aimg_stride + ((size_t)tile * 2 * (n2 / 8) + 2 * j) * 1024;
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                                 " [%0], [%1], %2, [%3], %4;"
                                 ::"r"(tc::smem_u32(stage(s))), "l"(asrc), "r"(abytes), "r"(mb), "l"(stream_pol)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                                 " [%0], [%1], %2, [%3], %4;"
                                 ::"r"(tc::smem_u32(stage(s) + ST2_ALO)), "l"(asrc + (size_t)(n2 / 8) * 1024),
                                 "r"(abytes), "r"(mb), "l"(stream_pol)
                                 : "memory");
                    for (int nb = 0; nb < nbk; ++nb) {
                        // rows pass ne2 + nb nb_u + rank hrow .. + hrow of both planes
                        const __nv_bfloat16* bsrc = A.bu + (size_t)fw * A.bu_stride + (size_t)j * 2 * img_u +
                                                    (size_t)(pass * ne2 + nb * nb_u + (int)rank * hrow) * 16;
                        const uint32_t dh = tc::smem_u32(stage(s) + ST2_B + (uint32_t)nb * hb);
                        const uint32_t dl = tc::smem_u32(stage(s) + ST2_B + (uint32_t)(nbk + nb) * hb);
                        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                     ::"r"(dh), "l"(bsrc), "r"(hb), "r"(mb)
                                     : "memory");
                        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                     ::"r"(dl), "l"(bsrc + img_u), "r"(hb), "r"(mb)
                                     : "memory");
                    }
                } else {
                    if (j == nU) {
                        // this CTA's |G|^2 slices of the item are written by its producers
                        if (!tc::mbar_wait(tc::smem_u32(&s_vready), vrp & 1u, kMaxTries)) {
                            err = true;
                            break;
                        }
                        ++vrp;
                    }
                    const uint32_t wbytes = (uint32_t)wrow * 64u, abytes = 2u * TP * 32 * 2;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(wbytes + abytes)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(tc::smem_u32(stage(s) + ST2_VB)),
                                 "l"(A.bw + (size_t)fw * A.bw_stride + (size_t)(j - nU) * img_w +
                                     (size_t)(pass * ne + (int)rank * wrow) * 32),
                                 "r"(wbytes), "r"(mb)
                                 : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(tc::smem_u32(stage(s))), "l"(vimg + (size_t)(j - nU) * (2 * TP * 32)), "r"(abytes),
                                 "r"(mb)
                                 : "memory");
                }
                if (++s == NST2) { s = 0; ph ^= 1u; }
                if (++j == per) {
                    j = 0;
                    if (++pass == npass) {
                        pass = 0;
                        if (++fw == A.F.n) { fw = 0; q += nq; }
                    }
                }
            }
            if (err || s_err) {
                s_err = 1;
                for (int x = (ql > NST2 ? ql - NST2 : 0); x < ql; ++x)
                    tc::mbar_wait(tc::smem_u32(&s_full[x % NST2]), (uint32_t)(x / NST2) & 1u, kMaxTries);
            }
        }
        __syncwarp();
    } else if (warp == NPROD / 32 && rank != 0) {
        // ------------------------------ relay (rank 1) ------------------------------
        if (lane == 0) {
            const uint32_t r_pfull = tc::mapa(tc::smem_u32(&s_pfull[0]), 0u);
            int s = 0;
            uint32_t ph = 0;
            for (int ql = 0; ql < total; ++ql) {
                if (!tc::mbar_wait(tc::smem_u32(&s_full[s]), ph, kMaxTries)) {
                    s_err = 1;
                    break;
                }
                if (s_err) break;
                tc::mbar_arrive_remote(r_pfull + 8u * (uint32_t)s);
                if (++s == NST2) { s = 0; ph ^= 1u; }
            }
        }
        __syncwarp();
    } else if (warp == NPROD / 32) {
        // ------------------------------ MMA issuer (rank 0) ------------------------------
        if (lane == 0) {
            const uint32_t id_u = tc::idesc_bf16_f32(256, (uint32_t)nb_u);
            const uint32_t id_v = tc::idesc_bf16_f32(256, (uint32_t)ne);
            int s = 0, j = 0;
            uint32_t acce = 0, accl = 0, ph = 0;
            bool err = false, issued = false;
            for (int q = 0; q < total && !err; ++q) {
                if (j == nU) {
                    // V overwrites the columns of the first N-block of U: both CTAs' part of the U
                    // epilogue there must be done
                    if (!tc::mbar_wait_cluster(tc::smem_u32(&s_acc_low), accl & 1u, kMaxTries)) { err = true; break; }
                    ++accl;
                } else if (j == 0 && q > 0) {
                    // a new U phase: both CTAs' V (or U) epilogue must have read the accumulator
                    if (!tc::mbar_wait_cluster(tc::smem_u32(&s_acc_empty), acce & 1u, kMaxTries)) { err = true; break; }
                    ++acce;
                }
                if (!tc::mbar_wait(tc::smem_u32(&s_full[s]), ph, kMaxTries)) { err = true; break; }
                if (!tc::mbar_wait_cluster(tc::smem_u32(&s_pfull[s]), ph, kMaxTries)) { err = true; break; }
                if (s_err) { err = true; break; }
                tc::fence_after();
                const uint32_t sa = tc::smem_u32(stage(s)), sal = sa + ST2_ALO, sb = sa + ST2_B;
                const uint64_t dah = tc::sdesc(sa, 2048, 128), dal = tc::sdesc(sal, 2048, 128);
                if (j < nU) {
                    const uint32_t acc = j > 0 ? 1u : 0u;
                    for (int nb = 0; nb < nbk; ++nb) {
                        const uint64_t dbh = tc::sdesc(sb + (uint32_t)nb * hb, 128, 256);
                        const uint64_t dbl = tc::sdesc(sb + (uint32_t)(nbk + nb) * hb, 128, 256);
                        const uint32_t d = tmem + (uint32_t)(nb * nb_u);
                        tc::mma_bf16_pair(d, dah, dbh, id_u, acc);
                        tc::mma_bf16_pair(d, dah, dbl, id_u, 1u);
                        tc::mma_bf16_pair(d, dal, dbh, id_u, 1u);
                    }
                } else {
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        const uint64_t vah = tc::sdesc(sa + 256u * kh, 128, 512);
                        const uint64_t val = tc::sdesc(sa + ST2_VALO + 256u * kh, 128, 512);
                        const uint64_t vb = tc::sdesc(sa + ST2_VB + 256u * kh, 128, 512);
                        tc::mma_bf16_pair(tmem, vah, vb, id_v, (j > nU || kh > 0) ? 1u : 0u);
                        tc::mma_bf16_pair(tmem, val, vb, id_v, 1u);
                    }
                }
                issued = true;
                tc::commit_pair(tc::smem_u32(&s_empty[s]));
                if (j == nU - 1 || j == per - 1) tc::commit_pair(tc::smem_u32(&s_acc_full));
                if (++s == NST2) { s = 0; ph ^= 1u; }
                if (++j == per) j = 0;
            }
            if (err) {
                s_err = 1;
                atomicAdd(A.counters + CNT_TC_TIMEOUT, 1u);
                if (issued) {
                    tc::commit_pair_local(tc::smem_u32(&s_drain));
                    tc::mbar_wait(tc::smem_u32(&s_drain), 0u, kMaxTries);
                }
            }
        }
        __syncwarp();
    } else {
        // -------------------------------- producers (both CTAs) --------------------------------
        const uint32_t p = (uint32_t)(tid & (TP - 1)), h = (uint32_t)(tid / TP);
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        const uint32_t cp = (uint32_t)((lane & 7) + 8 * warp), ch = (uint32_t)(lane >> 3);
        float2* gs = A.gscr + (size_t)blockIdx.x * n * TP;
        // the issuer's accumulator barriers (in rank 0), arrived on by both CTAs
        const uint32_t r_acc_empty = tc::mapa(tc::smem_u32(&s_acc_empty), 0u);
        const uint32_t r_acc_low = tc::mapa(tc::smem_u32(&s_acc_low), 0u);
        bool err = false;
        int qs = 0;
        uint32_t qph = 0;
        uint32_t accf = 0;
        auto slice = [&](auto&& consume) {
            const int s = qs;
            if (!err) err = !tc::mbar_wait(tc::smem_u32(&s_full[s]), qph, kMaxTries);
            err = __any_sync(0xffffffffu, err || s_err != 0);
            if (!err) consume(stage(s), stage(s) + ST2_ALO);
            __syncwarp();
            if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_empty[s]));
            if (++qs == NST2) { qs = 0; qph ^= 1u; }
        };
        auto acc_wait = [&]() {
            if (!err) err = !tc::mbar_wait(tc::smem_u32(&s_acc_full), accf & 1u, kMaxTries);
            ++accf;
            err = __any_sync(0xffffffffu, err);
            tc::fence_after();
        };
        auto arrive_issuer = [&](uint32_t caddr) {
            tc::fence_before();
            __syncwarp();
            if (lane == 0 && !err) tc::mbar_arrive_remote(caddr);
        };
        for (int q = q0; q < n_pairs; q += nq) {
            const int tile = tile_of(q);
            const int px = tile * TP + (int)p;
            const bool valid = px < G.npix && 2 * q + (int)rank < A.n_tiles;
            float acc_g = 0.f, acc_h = 0.f;
            for (int fw = 0; fw < A.F.n; ++fw) {
                const FreqC fc = A.F.f[fw];
                float fg_r = 0.f, fg_i = 0.f, fh = 0.f;
                for (int pass = 0; pass < npass; ++pass) {
                const int eb0 = pass * ne;
                for (int j = 0; j < nU; ++j)
                    slice([&](const unsigned char* ahi, const unsigned char* alo) {
                        consume_u(j * 8, cp, ch, ahi, alo, gs, vimg, want_h);
                    });
                if (want_h) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_vready));
                }
                err = tc::named_or(1, NPROD, err);
                if (err) break;
                const int nch = 4 * ((ne / 32 - (int)h + 3) / 4);
                const int nbu = ne2 > 256 ? ne2 / 2 : ne2, ebu = nbu / 2;
                auto ce0 = [&](int k) { return 32 * ((int)h + 4 * (k >> 2)) + 8 * (k & 3); };
                auto recol = [&](int e) { return (e / ebu) * nbu + e % ebu; };
                auto gload = [&](int k, float2 (&g)[8]) {
                    const int e0 = ce0(k);
#pragma unroll
                    for (int i = 0; i < 8; ++i) g[i] = gs[(size_t)(eb0 + e0 + i) * TP + p];
                };
                auto gchunk = [&](int k, const float2 (&g)[8], float& ar, float& ai) {
                    const int e0 = ce0(k);
                    float vr[8], vi[8];
                    tc::tmem_ld8(tmem + lane_off + (uint32_t)recol(e0), vr);
                    tc::tmem_ld8(tmem + lane_off + (uint32_t)(recol(e0) + ebu), vi);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        ar = fmaf(g[i].x, vr[i], fmaf(g[i].y, vi[i], ar));
                        ai = fmaf(g[i].x, vi[i], fmaf(-g[i].y, vr[i], ai));
                    }
                };
                bool low = false;
                auto release_low = [&]() {
                    arrive_issuer(r_acc_low);
                    low = true;
                };
                float2 ga[8], gb[8];
                if (nch > 0) gload(0, ga);
                acc_wait();
                float gr = 0.f, gi = 0.f;
                if (!err) {
                    for (int k = 0; k < nch; k += 2) {
                        if (!low && ce0(k) >= ebu) release_low();
                        gload(k + 1, gb);
                        gchunk(k, ga, gr, gi);
                        if (k + 2 < nch) gload(k + 2, ga);
                        gchunk(k + 1, gb, gr, gi);
                    }
                }
                if (!low) release_low();
                if (h > 0) {
                    s_red[0][h - 1][p] = gr;
                    s_red[1][h - 1][p] = gi;
                }
                err = tc::named_or(1, NPROD, err);
                if (err) break;
                if (h == 0) {
                    fg_r += (gr + s_red[0][0][p] + s_red[0][1][p] + s_red[0][2][p]) * fc.w2;
                    fg_i += (gi + s_red[1][0][p] + s_red[1][1][p] + s_red[1][2][p]) * fc.w2;
                }
                if (!want_h) {
                    arrive_issuer(r_acc_empty);
                    continue;
                }
                // V slices: the producers only pass the stage barriers (as in the single-CTA kernel)
                for (int j = 0; j < nV; ++j) slice([&](const unsigned char*, const unsigned char*) {});
                uint4 qa[2], qb[2];
                if (nch > 0) g2_load(vimg, eb0 + ce0(0), p, qa);
                acc_wait();
                float hh = 0.f;
                if (!err) {
                    for (int k = 0; k < nch; k += 2) {
                        g2_load(vimg, eb0 + ce0(k + 1), p, qb);
                        h_chunk(tmem + lane_off + (uint32_t)ce0(k), qa, hh);
                        if (k + 2 < nch) g2_load(vimg, eb0 + ce0(k + 2), p, qa);
                        h_chunk(tmem + lane_off + (uint32_t)ce0(k + 1), qb, hh);
                    }
                }
                arrive_issuer(r_acc_empty);
                if (h > 0) s_red[2][h - 1][p] = hh;
                err = tc::named_or(1, NPROD, err);
                if (err) break;
                if (h == 0) fh += (hh + s_red[2][0][p] + s_red[2][1][p] + s_red[2][2][p]) * fc.w4;
                }   // passes
                if (err) break;
                if (h == 0) {
                    if (valid && A.g_out) A.g_out[(size_t)fw * G.npix + px] = make_float2(fg_r, fg_i);
                    if (valid && A.h_out) A.h_out[(size_t)fw * G.npix + px] = fh;
                    acc_g += fg_r;
                    acc_h += fh;
                }
            }
            if (err) break;
            if (valid && h == 0) {
                if (A.gsum) A.gsum[px] = acc_g;
                if (A.hsum) A.hsum[px] = acc_h;
            }
        }
    }
    tc::fence_before();
    tc::cluster_sync();   // the peer is done with this CTA's shared memory and barriers
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc_pair(tmem, A.tmem_cols);
}
}  // namespace

// rings of 64..256 elements in multiples of 64 in one pass over the elements of U and V,
// and of 512, 768 and 1024 elements in passes of 256
bool tc_adjoint_supported(int n_elem) {
    return (n_elem >= 64 && n_elem <= 256 && n_elem % 64 == 0) || (n_elem % 256 == 0 && n_elem >= 512 && n_elem <= 1024);
}


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

size_t tc_aimage_elems(int n_elem, int npix) {
    return (size_t)((npix + TP - 1) / TP) * 2 * (size_t)(2 * n_elem / 8) * 1024;
}

cudaError_t launch_tables_images(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F, void* aimg,
                                 cudaStream_t s) {
    if (!tc_adjoint_supported(G.n_elem) || !tables || !c || !aimg) return cudaErrorInvalidValue;
    const int n_tiles = (G.npix + TP - 1) / TP;
    const long long blocks = (long long)n_tiles * (G.n_elem / 16);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_tables_images<<<(int)blocks, 256, 0, s>>>(G, tables, c, F, (__nv_bfloat16*)aimg,
                                                tc_aimage_elems(G.n_elem, G.npix));
    return cudaGetLastError();
}

namespace {
// gsum = sum over the set's frequencies of Re g, hsum of H, added in frequency order (the
// order a CTA taking all frequencies of its tile in turn would use).
__global__ void k_adjoint_sums(const float2* __restrict__ fpart, int n_freq, int npix, float* __restrict__ gsum,
                               float* __restrict__ hsum) {
    for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < npix; px += gridDim.x * blockDim.x) {
        float g = 0.f, h = 0.f;
        for (int fw = 0; fw < n_freq; ++fw) {
            const float2 v = fpart[(size_t)fw * npix + px];
            g += v.x;
            h += v.y;
        }
        if (gsum) gsum[px] = g;
        if (hsum) hsum[px] = h;
    }
}
}  // namespace

cudaError_t launch_adjoint_tc(const GeoDev& G, const void* aimg, const FreqSet& F, const void* images, float2* gscr,
                              int n_ctas, float2* g_out, float* h_out, float* gsum, float* hsum, uint32_t* counters,
                              cudaStream_t s, int variant) {
    const int n = G.n_elem;
    if (!tc_adjoint_supported(n) || !aimg) return cudaErrorInvalidValue;
    TcArgs A;
    A.G = G;
    A.F = F;
    A.aimg = (const __nv_bfloat16*)aimg;
    A.aimg_stride = tc_aimage_elems(n, G.npix);
    A.bu = (const __nv_bfloat16*)images;
    A.bu_stride = tc_b_images_bytes(n) / 2;
    A.bw = A.bu + (size_t)(2 * n) * (2 * n) * 2;
    A.bw_stride = A.bu_stride;
    A.gscr = gscr;
    A.vimg = (__nv_bfloat16*)(gscr + (size_t)RB_TC_MAX_CTAS * n * TP);   // after the G scratch
    A.g_out = g_out;
    A.h_out = h_out;
    A.gsum = gsum;
    A.hsum = hsum;
    A.fpart = nullptr;
    A.counters = counters;
    A.n_tiles = (G.npix + TP - 1) / TP;
    A.n_e = n < 256 ? n : 256;
    A.want_h = (h_out || hsum) ? 1 : 0;
    A.npass = n / A.n_e;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * A.n_e)) cols <<= 1;
    A.tmem_cols = cols;
    cudaError_t e;
    // variant 1: CTA pairs (8 stages of 24 KB); 0 and 2: one CTA per tile (5 stages of 40 KB);
    // either way most of the SM's shared memory, so one CTA (one TMEM owner) per SM
    const int n_pairs = (A.n_tiles + 1) / 2;
    if (variant == 1 && n_ctas >= 2) {
        const int sm2 = NST2 * (int)ST2_BYTES;
        const int grid2 = 2 * (n_ctas / 2 < n_pairs ? n_ctas / 2 : n_pairs);
        if (A.npass == 1) {
            e = cudaFuncSetAttribute(k_adjoint_tc2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
            if (e != cudaSuccess) return e;
            k_adjoint_tc2<false><<<grid2, NTHR_A, sm2, s>>>(A);
        } else {
            e = cudaFuncSetAttribute(k_adjoint_tc2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
            if (e != cudaSuccess) return e;
            k_adjoint_tc2<true><<<grid2, NTHR_A, sm2, s>>>(A);
        }
        return cudaGetLastError();
    }
    // the CTAs take (tile, frequency) items in turn, so the sums over the set go through
    // the per-frequency buffer that follows the per-CTA scratch in the workspace
    if (gsum || hsum)
        A.fpart = (float2*)(A.vimg + (size_t)RB_TC_MAX_CTAS * n * 256);
    const int sm = NST * (int)ST_BYTES;
    const int n_items = A.n_tiles * F.n;
    const int grid = n_ctas < n_items ? n_ctas : n_items;
    if (A.npass == 1) {
        e = cudaFuncSetAttribute(k_adjoint_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_adjoint_tc<false><<<grid, NTHR_A, sm, s>>>(A);
    } else {
        e = cudaFuncSetAttribute(k_adjoint_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_adjoint_tc<true><<<grid, NTHR_A, sm, s>>>(A);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || !A.fpart) return e;
    k_adjoint_sums<<<(G.npix + 255) / 256, 256, 0, s>>>(A.fpart, F.n, G.npix, gsum, hsum);
    return cudaGetLastError();
}

// ===========================================================================
// Born forward on the tensor cores:  d[e][r] = w^2 sum_x G_e(x) G_r(x) m(x)
// Real form over K = pixels: rows e' = 2e + {0: Re, 1: -Im} of A = conj(G) m and
// columns r' = 2r + {0, 1} of B = conj(G) give D = A B^T (2n x 2n, symmetric) =
// the real form of conj(d), from which
//   Re d = D[2e][2r] - D[2e+1][2r+1],  Im d = -(D[2e][2r+1] + D[2e+1][2r]).
// Both operands come from the adjoint's A image (layout of aimg_put4), read MN-major:
// a core matrix there is 8 pixels (K) x 8 consecutive r' (16 bytes each), and a
// 16-pixel K slice of all r' rows is one 2-D TMA box per plane.  CTA (i, s):
// 128-row block i of D over pixel split s, the needed column blocks in TMEM;
// column blocks below the diagonal are skipped (symmetry).  Partial D blocks go to
// global memory and a second kernel sums the splits in order.
// ===========================================================================
namespace {

constexpr int FMAXB = 16;  // max row blocks (2n / 128, n <= 1024)
constexpr int FMAXG = 4;   // max column groups of two 256-column blocks (2n / 512)
constexpr int FMAXP = 40;  // max (row block, column group) pairs (40 for n = 1024)
constexpr int FBOX_MAX = 32;   // rows (of 8 r') per TMA box, at most
constexpr uint32_t ST_FB = 8192u;   // forward stage: A hi (4 KB), A lo (4 KB), then B hi and B lo

struct FwdArgs {
    GeoDev G;
    FreqC F;
    const float* m;
    float* partial;            // [cta][128][2n] fp32 (only needed columns written)
    int n_mb;                  // row blocks
    int nbn, nb;               // column blocks and their width
    // work pairs: row block p_i with the column blocks [p_jb, p_je) (at most two, so the
    // accumulators fit TMEM), each split over pixel ranges
    int n_pairs;
    int p_i[FMAXP], p_jb[FMAXP], p_je[FMAXP];
    int splits[FMAXP];         // splits per pair
    int cta0[FMAXP + 1];       // first CTA of each pair
    int pidx[FMAXB][FMAXG];    // pair of (row block, column group of two blocks)
    uint32_t tmem_cols;
    uint32_t* counters;
    int fbox;                  // rows per TMA box of the B rows: divides every pair's loaded rows
};

__host__ __device__ __forceinline__ int jmin_of(int i, int nb) { return (128 * i) / nb; }

// Forward kernel: warp-specialised pipeline over K = 16 pixel slices.
//   warps 0..7  producers: thread u takes the 16-byte row (8 r', one pixel) u of the
//               row block's A slice: B rows 128 i .. 128 i + 127 scaled by m(x) and
//               re-split into hi / lo, once the slice's B has landed; then the epilogue;
//   warp 8      MMA issuer; warp 9 loader (TMA boxes of the rows [col0, 2n) of the
//               slice, hi and lo planes).
// SEP: some pairs load their row block's own rows separately (rings above 256 elements);
// without it every pair finds them among its B rows and the test compiles away.
template <bool SEP>
__global__ void __launch_bounds__(NTHR_F, 1) k_forward_tc(FwdArgs A, const __grid_constant__ CUtensorMap tmap,
                                                         const __grid_constant__ CUtensorMap tmap16) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_full_a[NST], s_full_b[NST], s_empty[NST], s_acc_full;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_err;
    const GeoDev& G = A.G;
    const int n = G.n_elem, n2 = 2 * n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int pq = 0;
    while (pq + 1 < A.n_pairs && (int)blockIdx.x >= A.cta0[pq + 1]) ++pq;
    const int i = A.p_i[pq], jb = A.p_jb[pq], je = A.p_je[pq];
    const int sp = (int)blockIdx.x - A.cta0[pq];
    const int S = A.splits[pq];
    const int col0 = jb * A.nb, col1 = je * A.nb;       // needed columns (= B rows loaded)
    const int rcn = n2 / 8, rc0 = col0 / 8;             // rows of 8 r' per plane; first one loaded
    const int nrow = (col1 - col0) / 8;                 // rows loaded per plane (a multiple of fbox)
    const uint32_t plane_bytes = (uint32_t)nrow * 256u;
    // the row block's own 16 rows (the A operand before scaling by m): inside the loaded B
    // rows, or loaded separately into the A area of the stage
    const bool own_in = !SEP || (16 * i >= rc0 && 16 * i + 16 <= rc0 + nrow);
    const uint32_t tx_bytes = 2u * plane_bytes + (own_in ? 0u : 2u * 16u * 256u);
    const int n_tiles = (G.npix + TP - 1) / TP;
    const int nsl_all = n_tiles * 8;
    const int cps = (nsl_all + S - 1) / S;
    const int sbeg = min(nsl_all, sp * cps), send = min(nsl_all, sbeg + cps);
    const int nq = send - sbeg;
    if (tid == 0) {
        for (int k = 0; k < NST; ++k) {
            tc::mbar_init(tc::smem_u32(&s_full_a[k]), NPROD_F / 32);
            tc::mbar_init(tc::smem_u32(&s_full_b[k]), 1);
            tc::mbar_init(tc::smem_u32(&s_empty[k]), 1);
        }
        tc::mbar_init(tc::smem_u32(&s_acc_full), 1);
        s_err = 0;
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&s_tmem), A.tmem_cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    auto stage = [&](int k) { return smem + (size_t)k * ST_BYTES; };

    if (warp == NPROD_F / 32 + 1) {
        // ------------------------------ loader ------------------------------
        if (lane == 0) {
            int ql = 0;
            bool err = false;
            const uint64_t tm = reinterpret_cast<uint64_t>(&tmap);
            const uint64_t tm16 = reinterpret_cast<uint64_t>(&tmap16);   // 16-row boxes: a row block's own rows
            for (; ql < nq; ++ql) {
                const int k = ql % NST;
                if (ql >= NST && !tc::mbar_wait(tc::smem_u32(&s_empty[k]), (uint32_t)((ql / NST) - 1) & 1u, kMaxTries)) {
                    err = true;
                    break;
                }
                if (s_err) break;
                const int sg = sbeg + ql, t = sg >> 3, x = (sg & 7) * 128;
                const uint32_t mb = tc::smem_u32(&s_full_b[k]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx_bytes)
                             : "memory");
                for (int hl = 0; hl < 2; ++hl) {
                    for (int b = 0; b < nrow / A.fbox; ++b) {
                        const uint32_t dst = tc::smem_u32(stage(k) + ST_FB + hl * plane_bytes + (uint32_t)(b * A.fbox) * 256u);
                        const int y = (t * 2 + hl) * rcn + rc0 + b * A.fbox;
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                            ::"r"(dst), "l"(tm), "r"(x), "r"(y), "r"(mb)
                            : "memory");
                    }
                    if (!own_in) {
                        const uint32_t dst = tc::smem_u32(stage(k) + hl * ST_ALO);
                        const int y = (t * 2 + hl) * rcn + 16 * i;
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                            ::"r"(dst), "l"(tm16), "r"(x), "r"(y), "r"(mb)
                            : "memory");
                    }
                }
            }
            if (err || s_err) {
                s_err = 1;
                for (int x = (ql > NST ? ql - NST : 0); x < ql; ++x)
                    tc::mbar_wait(tc::smem_u32(&s_full_b[x % NST]), (uint32_t)(x / NST) & 1u, kMaxTries);
            }
        }
        __syncwarp();
    } else if (warp == NPROD_F / 32) {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            // both operands MN-major (transpose bits 15 and 16): LBO = stride between the
            // two 8-pixel K cores (128 B), SBO = stride between 8-r' cores (256 B)
            const uint32_t id = tc::idesc_bf16_f32(128, (uint32_t)A.nb) | (1u << 15) | (1u << 16);
            int last = -1;
            bool err = false;
            for (int q = 0; q < nq && !err; ++q) {
                const int k = q % NST;
                const uint32_t ph = (uint32_t)(q / NST) & 1u;
                if (!tc::mbar_wait(tc::smem_u32(&s_full_a[k]), ph, kMaxTries)) { err = true; break; }
                if (!tc::mbar_wait(tc::smem_u32(&s_full_b[k]), ph, kMaxTries)) { err = true; break; }
                if (s_err) { err = true; break; }
                tc::fence_after();
                const uint32_t sa = tc::smem_u32(stage(k)), sb = sa + ST_FB;
                const uint64_t dah = tc::sdesc(sa, 128, 256), dal = tc::sdesc(sa + ST_ALO, 128, 256);
                for (int j = jb; j < je; ++j) {
                    const uint32_t boff = (uint32_t)((j * A.nb) / 8 - rc0) * 256u;
                    const uint64_t dbh = tc::sdesc(sb + boff, 128, 256);
                    const uint64_t dbl = tc::sdesc(sb + plane_bytes + boff, 128, 256);
                    const uint32_t d = tmem + (uint32_t)((j - jb) * A.nb);
                    tc::mma_bf16(d, dah, dbh, id, q > 0 ? 1u : 0u);
                    tc::mma_bf16(d, dah, dbl, id, 1u);
                    tc::mma_bf16(d, dal, dbh, id, 1u);
                }
                tc::commit(tc::smem_u32(&s_empty[k]));
                if (q == nq - 1) tc::commit(tc::smem_u32(&s_acc_full));
                last = q;
            }
            if (err) {
                s_err = 1;
                atomicAdd(A.counters + CNT_TC_TIMEOUT, 1u);
                if (last >= 0) tc::mbar_wait(tc::smem_u32(&s_empty[last % NST]), (uint32_t)(last / NST) & 1u, kMaxTries);
            }
        }
        __syncwarp();
    } else {
        // -------------------------------- producers --------------------------------
        // thread tid: row rl = tid / 16 of 8 r' (of the row block's 16), K core pc = (tid / 8) % 2,
        // pixel row x8 = tid % 8 of that core
        const int rl = tid >> 4, pc = (tid >> 3) & 1, x8 = tid & 7;
        const uint32_t aoff = (uint32_t)(rl * 256 + pc * 128 + x8 * 16);
        // source of this thread's 16 bytes: the B rows, or the A area itself (scaled in place)
        const uint32_t soff = own_in ? ST_FB + (uint32_t)((16 * i - rc0 + rl) * 256 + pc * 128 + x8 * 16) : aoff;
        const uint32_t slo = own_in ? plane_bytes : ST_ALO;
        bool err = false;
        auto load_m = [&](int q) -> float {
            if (q >= nq) return 0.f;
            const int px = (sbeg + q) * 16 + pc * 8 + x8;
            return px < G.npix ? __ldg(A.m + px) : 0.f;
        };
        float mnext = load_m(0);
        for (int q = 0; q < nq; ++q) {
            const int k = q % NST;
            const uint32_t ph = (uint32_t)(q / NST) & 1u;
            const float mm = mnext;
            mnext = load_m(q + 1);
            if (!err && q >= NST) err = !tc::mbar_wait(tc::smem_u32(&s_empty[k]), ph ^ 1u, kMaxTries);
            if (!err) err = !tc::mbar_wait(tc::smem_u32(&s_full_b[k]), ph, kMaxTries);
            err = __any_sync(0xffffffffu, err || s_err != 0);
            if (!err) {
                const unsigned char* src = stage(k) + soff;
                const uint4 vh = *(const uint4*)src, vl = *(const uint4*)(src + slo);
                const uint32_t hw[4] = {vh.x, vh.y, vh.z, vh.w}, lw[4] = {vl.x, vl.y, vl.z, vl.w};
                uint32_t oh[4], ol[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float x0 = (__bfloat162float(__ushort_as_bfloat16((unsigned short)(hw[t] & 0xffff))) +
                                      __bfloat162float(__ushort_as_bfloat16((unsigned short)(lw[t] & 0xffff)))) * mm;
                    const float x1 = (__bfloat162float(__ushort_as_bfloat16((unsigned short)(hw[t] >> 16))) +
                                      __bfloat162float(__ushort_as_bfloat16((unsigned short)(lw[t] >> 16)))) * mm;
                    __nv_bfloat16 h0, l0, h1, l1;
                    tc::split_bf16(x0, h0, l0);
                    tc::split_bf16(x1, h1, l1);
                    oh[t] = pack2(h0, h1);
                    ol[t] = pack2(l0, l1);
                }
                *(uint4*)(stage(k) + aoff) = make_uint4(oh[0], oh[1], oh[2], oh[3]);
                *(uint4*)(stage(k) + ST_ALO + aoff) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0 && !err) tc::mbar_arrive(tc::smem_u32(&s_full_a[k]));
        }
        // epilogue: this CTA's partial D block (128 rows x needed columns) to global memory
        if (!err && nq > 0) err = !tc::mbar_wait(tc::smem_u32(&s_acc_full), 0u, kMaxTries);
        err = __any_sync(0xffffffffu, err || s_err != 0);
        tc::fence_after();
        if (!err) {
            const int row = tid & 127, g = tid >> 7;
            const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
            float* out = A.partial + ((size_t)blockIdx.x * 128 + row) * n2;
            int cnum = 0;
            for (int cb = col0; cb < col1; cb += 32, ++cnum) {
                if ((cnum & 1) != g) continue;
                float v[32];
                if (nq > 0) {
                    tc::tmem_ld32(tmem + lane_off + (uint32_t)(cb - col0), v);
                } else {
#pragma unroll
                    for (int t = 0; t < 32; ++t) v[t] = 0.f;
                }
#pragma unroll
                for (int t = 0; t < 32; t += 4) *(float4*)(out + cb + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, A.tmem_cols);
}

// d = w^2 (sum over splits of the partial D blocks, symmetric lookup), and
// per-block partial sums of W |d|^2.
// d = w^2 (sum over splits of the partial D blocks), and per-block partial sums of
// W |d|^2.  D and d are symmetric, and for e <= r the 2 x 2 block of D at (2e, 2r) lies in
// a computed block (on or above the block diagonal), so thread (e, r), e <= r, reads it
// row-wise (consecutive threads, consecutive r: coalesced) and writes d[e][r] and d[r][e].
__global__ void k_forward_tc_reduce(FwdArgs A, float2* __restrict__ d_out, const uint8_t* __restrict__ w,
                                    double* __restrict__ den_part) {
    const int n = A.G.n_elem, n2 = 2 * n;
    double acc = 0.0;
    const long long total = (long long)n * n;
    for (long long jj = blockIdx.x * (long long)blockDim.x + threadIdx.x; jj < total;
         jj += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(jj / n), r = (int)(jj % n);
        if (e > r) continue;
        const int i = (2 * e) >> 7, row = (2 * e) & 127;
        const int pq = A.pidx[i][((2 * r) / A.nb) >> 1];
        float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f);   // D[2e][2r..2r+1], D[2e+1][2r..2r+1]
        for (int sp = 0; sp < A.splits[pq]; ++sp) {
            const float* blk = A.partial + ((size_t)(A.cta0[pq] + sp) * 128 + row) * n2 + 2 * r;
            const float2 a0 = *(const float2*)blk, a1 = *(const float2*)(blk + n2);
            d0.x += a0.x;
            d0.y += a0.y;
            d1.x += a1.x;
            d1.y += a1.y;
        }
        // the image rows 2r + 1 hold -Im G_r (the conjugate, as the adjoint uses it), so the
        // product of the two images is conj(d): Re d as is, Im d negated
        const float dre = (d0.x - d1.y) * A.F.w2;
        const float dim = -(d0.y + d1.x) * A.F.w2;
        const size_t er = (size_t)e * n + r, re = (size_t)r * n + e;
        if (d_out) {
            d_out[er] = make_float2(dre, dim);
            if (e != r) d_out[re] = make_float2(dre, dim);
        }
        if (w) {
            const int cnt = (w[er] ? 1 : 0) + ((e != r && w[re]) ? 1 : 0);
            if (cnt) acc += cnt * ((double)dre * dre + (double)dim * dim);
        }
    }
    if (den_part) {
        __shared__ double sred[256];
        sred[threadIdx.x] = acc;
        __syncthreads();
        for (int k = blockDim.x / 2; k > 0; k >>= 1) {
            if (threadIdx.x < k) sred[threadIdx.x] += sred[threadIdx.x + k];
            __syncthreads();
        }
        if (threadIdx.x == 0) den_part[blockIdx.x] = sred[0];
    }
}

FwdArgs make_fwd_args(const GeoDev& G, const FreqC& F, const float* m, float* partial, int n_ctas,
                      uint32_t* counters) {
    FwdArgs A;
    A.G = G;
    A.F = F;
    A.m = m;
    A.partial = partial;
    A.counters = counters;
    const int n2 = 2 * G.n_elem;
    A.n_mb = n2 / 128;
    A.nbn = (n2 + 255) / 256;
    A.nb = n2 / A.nbn;
    // pairs (row block i, column blocks [jb, je)): blocks from the diagonal one on, in
    // groups of two (group g holds blocks 2g and 2g + 1)
    A.n_pairs = 0;
    for (int i = 0; i < A.n_mb; ++i) {
        for (int g = 0; g < FMAXG; ++g) A.pidx[i][g] = -1;
        const int jmin = jmin_of(i, A.nb);
        for (int g = jmin / 2; 2 * g < A.nbn; ++g) {
            const int q = A.n_pairs++;
            A.p_i[q] = i;
            A.p_jb[q] = 2 * g > jmin ? 2 * g : jmin;
            A.p_je[q] = 2 * g + 2 < A.nbn ? 2 * g + 2 : A.nbn;
            A.pidx[i][g] = q;
        }
    }
    // TMEM: the widest pair, two blocks (one when there is only one)
    uint32_t cols = 32;
    while (cols < (uint32_t)((A.nbn > 1 ? 2 : 1) * A.nb)) cols <<= 1;
    A.tmem_cols = cols;
    // splits per pair: equal.  A pixel slice costs about the same on every pair, whether
    // it issues MMAs for one column block or two (the operand delivery and producer work
    // per slice, not the tensor pipe, set the pace), so splits in proportion to the
    // column blocks left the pairs with one block idle half the time.
    int c0 = 0;
    for (int q = 0; q < A.n_pairs; ++q) {
        int sq = n_ctas / A.n_pairs;
        if (sq < 1) sq = 1;
        A.splits[q] = sq;
        A.cta0[q] = c0;
        c0 += sq;
    }
    A.cta0[A.n_pairs] = c0;
    // TMA box height of the B rows: the largest power of two up to FBOX_MAX dividing every
    // pair's loaded rows (a row block's own 16 rows, where loaded apart, use 16-row boxes)
    A.fbox = FBOX_MAX;
    for (int q = 0; q < A.n_pairs; ++q) {
        const int nrow = (A.p_je[q] - A.p_jb[q]) * A.nb / 8;
        while (nrow % A.fbox != 0) A.fbox >>= 1;
    }
    return A;
}

}  // namespace

size_t tc_forward_partial_bytes(int n_elem, int n_ctas) {
    return (size_t)(n_ctas + FMAXP) * 128 * (2 * (size_t)n_elem) * sizeof(float);
}

namespace {

// The forward kernel of one frequency on s; its arguments (which the reduce takes too) in *out.
cudaError_t forward_tc_kernel(const GeoDev& G, const void* aimg, const FreqC& F, const float* m, float* partial,
                              int n_ctas, uint32_t* counters, cudaStream_t s, FwdArgs* out) {
    if (!tc_adjoint_supported(G.n_elem) || !aimg) return cudaErrorInvalidValue;
    const FwdArgs A = make_fwd_args(G, F, m, partial, n_ctas, counters);
    // the A image of this frequency as a 2-D tensor: rows of 8 r' x 128 pixels (1024 bf16),
    // (tile, plane, row) major; boxes of 128 elements (one 16-pixel slice) x fbox rows
    const int rcn = 2 * G.n_elem / 8;
    const int n_tiles = (G.npix + TP - 1) / TP;
    CUtensorMap tmap, tmap16;
    if (A.fbox < 1 || !tc::encode_tmap_2d(&tmap, aimg, 1024, (uint64_t)n_tiles * 2 * rcn, 2048, 128, (uint32_t)A.fbox))
        return cudaErrorUnknown;
    if (!tc::encode_tmap_2d(&tmap16, aimg, 1024, (uint64_t)n_tiles * 2 * rcn, 2048, 128, 16u)) return cudaErrorUnknown;
    const int sm = NST * (int)ST_BYTES;
    bool sep = false;
    for (int q = 0; q < A.n_pairs; ++q) {
        const int rc0 = A.p_jb[q] * A.nb / 8, nrow = (A.p_je[q] - A.p_jb[q]) * A.nb / 8;
        sep = sep || !(16 * A.p_i[q] >= rc0 && 16 * A.p_i[q] + 16 <= rc0 + nrow);
    }
    cudaError_t e;
    if (sep) {
        e = cudaFuncSetAttribute(k_forward_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_forward_tc<true><<<A.cta0[A.n_pairs], NTHR_F, sm, s>>>(A, tmap, tmap16);
    } else {
        e = cudaFuncSetAttribute(k_forward_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_forward_tc<false><<<A.cta0[A.n_pairs], NTHR_F, sm, s>>>(A, tmap, tmap16);
    }
    *out = A;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward_tc(const GeoDev& G, const void* aimg, const FreqC& F, const float* m, float* partial,
                              int n_ctas, float2* d_out, const uint8_t* w, double* den_part, uint32_t* counters,
                              cudaStream_t s) {
    FwdArgs A;
    cudaError_t e = forward_tc_kernel(G, aimg, F, m, partial, n_ctas, counters, s, &A);
    if (e != cudaSuccess) return e;
    k_forward_tc_reduce<<<256, 256, 0, s>>>(A, d_out, w, den_part);
    return cudaGetLastError();
}

cudaError_t launch_forward_tc_overlap(const GeoDev& G, const void* aimg, const FreqC& F, const float* m,
                                      float* partial, int n_ctas, float2* d_out, const uint8_t* w, double* den_part,
                                      uint32_t* counters, cudaStream_t s, cudaStream_t r, cudaEvent_t fwd_done,
                                      cudaEvent_t red_done) {
    FwdArgs A;
    cudaError_t e = forward_tc_kernel(G, aimg, F, m, partial, n_ctas, counters, s, &A);
    if (e == cudaSuccess) e = cudaEventRecord(fwd_done, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r, fwd_done, 0);
    if (e != cudaSuccess) return e;
    k_forward_tc_reduce<<<256, 256, 0, r>>>(A, d_out, w, den_part);
    e = cudaGetLastError();
    return e == cudaSuccess ? cudaEventRecord(red_done, r) : e;
}
