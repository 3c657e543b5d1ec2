// Internal definitions shared by the CUDA translation units of librb.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rb.h"

#define RB_PI_F 3.14159265358979323846f
#define RB_PI_D 3.14159265358979323846

// ---------------------------------------------------------------------------
// Device-side geometry, built once per call on the host.
// ---------------------------------------------------------------------------
struct GeoDev {
    int n_elem, nx, ny, n_rays, max_steps;
    int npix;
    float h, inv_h, cxg, cyg;   // cxg = (nx - 1) / 2
    float fxmax, fymax;         // nx - 1, ny - 1 as floats
    float h_hi, h_lo;           // h as a float pair
    float ds, R, R2;
    float inv_cref, c_ref;
    float inv_cref_lo;          // 1 / c_ref - inv_cref
    float j_floor;              // h / 4
    double R_d, ds_d, c_ref_d, h_d;
    long long r2max;            // support test on (2ix-(nx-1))^2 + (2iy-(ny-1))^2
    const float4* elem_xy;      // [n_elem] element positions as float pairs {x_hi, x_lo, y_hi, y_lo}
};

// Per-frequency constants of the Green's function (host-computed in double).
struct FreqC {
    double f_d;           // f [Hz]
    float f_hi, f_lo;     // f as a float pair
    float kf_hi, kf_lo;   // f / c_ref as a float pair  [cycles per metre]
    float w_isqrt;        // 1 / sqrt(w)
    float a_abs;          // K_a f_MHz^y: amplitude decay per unit alpha0 integral
    float disp_cyc;       // dispersion phase per unit alpha0 integral, in cycles
    float w2;             // w^2
    float w4;             // w^4
};

struct FreqSet {
    int n;
    FreqC f[RB_MAX_FREQ];
};

// ---------------------------------------------------------------------------
// Float-pair ("double-float") helpers: value = hi + lo, |lo| <= ulp(hi)/2.
// Written from the standard error-free transformations (Knuth TwoSum,
// Dekker FastTwoSum, FMA-based TwoProduct).
// ---------------------------------------------------------------------------
struct DF { float hi, lo; };

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    DF p = df_two_prod(a.hi, b.hi);
    float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_fast_two_sum(p.hi, lo);
}
__device__ __forceinline__ DF df_sqr(DF a) {
    DF p = df_two_prod(a.hi, a.hi);
    float lo = __fmaf_rn(2.0f * a.hi, a.lo, p.lo);
    return df_fast_two_sum(p.hi, lo);
}
__device__ __forceinline__ DF df_sqrt(DF a) {  // a > 0
    // one Newton correction of s = sqrt(a.hi); the correction is below ulp(s), so an
    // approximate 1 / (2 s) leaves the pair accurate to ~2^-46 relative
    float s = sqrtf(a.hi);
    float r = __fadd_rn(__fmaf_rn(-s, s, a.hi), a.lo);
    float e = r * (0.5f * rsqrtf(a.hi));
    return df_fast_two_sum(s, e);
}
__host__ __device__ __forceinline__ DF df_from_double(double v) {
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    return {hi, lo};
}

// Pixel-centre coordinate (k - centre) * h as a float pair, k - centre exact.
__device__ __forceinline__ DF df_pixel_coord(int idx, float centre, float h_hi, float h_lo) {
    float k = (float)idx - centre;
    DF p = df_two_prod(k, h_hi);
    return df_fast_two_sum(p.hi, __fmaf_rn(k, h_lo, p.lo));
}

// ---------------------------------------------------------------------------
// Order-preserving float <-> uint32 map for first-arrival keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f2key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

#define RB_HOLE 0xffffffffu

// ---------------------------------------------------------------------------
// Green's function of Eqs. 4-5 for one gridded entry, pixel and frequency.
//   G = sqrt(c(x) / (8 pi w J)) exp(-a_abs L) exp(i 2 pi [f T + disp L + 1/8 - kappa/4])
// with T = |x - x_t| / c_ref + T_res, J = max(|q|, h/4).  The phase in cycles
// keeps f |x - x_t| / c_ref as a float pair so that its fractional part is
// exact to ~1e-9 cycles before the final sincospi.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 green_eval(const rb_cell& rec, float c_px, DF dist, const FreqC& F,
                                             float j_floor) {
    if (rec.tkey == RB_HOLE) return make_float2(0.f, 0.f);
    const float tres = key2f(rec.tkey);
    const int kappa = (int)(rec.tag & 0xffu);
    DF P = df_mul(DF{F.kf_hi, F.kf_lo}, dist);
    float base = __fsub_rn(P.hi, rintf(P.hi));
    float cyc = base + P.lo + F.f_hi * tres + F.disp_cyc * rec.l + 0.125f - 0.25f * (float)(kappa & 3);
    cyc -= rintf(cyc);
    // |2 pi cyc| <= pi: the hardware sine / cosine are accurate to ~4e-7 absolute there
    float s, co;
    __sincosf((2.0f * RB_PI_F) * cyc, &s, &co);
    const float J = fmaxf(fabsf(rec.q), j_floor);
    const float amp = sqrtf(c_px) * rsqrtf((8.0f * RB_PI_F) * J) * F.w_isqrt * __expf(-F.a_abs * rec.l);
    return make_float2(amp * co, amp * s);
}

// Synthesis record of one gridded entry (element r, pixel x): everything of the
// Green's function that does not depend on the frequency, in 16 bytes:
//   x, y = T = |x - x_r| / c_ref + T_res as a float pair [s],
//   z    = L (>= 0), its sign bit carrying bit 0 of kappa mod 4,
//   w    = A0 = sqrt(c(x) / (8 pi J)), its sign bit carrying bit 1 of kappa mod 4.
// A hole is all zeros (A0 = 0).
__device__ __forceinline__ float4 synth_record(const rb_cell& rec, float c_px, DF dist, float inv_cref,
                                               float inv_cref_lo, float j_floor) {
    if (rec.tkey == RB_HOLE) return make_float4(0.f, 0.f, 0.f, 0.f);
    const DF T = df_add(df_mul(dist, DF{inv_cref, inv_cref_lo}), DF{key2f(rec.tkey), 0.f});
    const uint32_t kappa = rec.tag & 3u;
    const float J = fmaxf(fabsf(rec.q), j_floor);
    const float A0 = sqrtf(c_px) * rsqrtf((8.0f * RB_PI_F) * J);
    const float L = __uint_as_float(__float_as_uint(fabsf(rec.l)) | ((kappa & 1u) << 31));
    const float Aw = __uint_as_float(__float_as_uint(A0) | ((kappa >> 1) << 31));
    return make_float4(T.hi, T.lo, L, Aw);
}

// The Green's function of Eqs. 4-5 at one frequency from a synthesis record:
//   G = A0 w^-1/2 exp(-a_abs L) exp(i 2 pi [f T + disp L + 1/8]) (-i)^kappa.
__device__ __forceinline__ float2 green_srec(float4 sr, const FreqC& F) {
    const uint32_t bz = __float_as_uint(sr.z), bw = __float_as_uint(sr.w);
    const float L = __uint_as_float(bz & 0x7fffffffu), A0 = __uint_as_float(bw & 0x7fffffffu);
    const DF P = df_mul(DF{F.f_hi, F.f_lo}, DF{sr.x, sr.y});
    float cyc = __fsub_rn(P.hi, rintf(P.hi)) + P.lo + fmaf(F.disp_cyc, L, 0.125f);
    cyc -= rintf(cyc);
    float s, c;
    __sincosf((2.0f * RB_PI_F) * cyc, &s, &c);
    const float amp = A0 * F.w_isqrt * __expf(-F.a_abs * L);
    float re = (bz >> 31) ? s : c, im = (bz >> 31) ? -c : s;   // kappa bit 0: times -i
    if (bw >> 31) {                                              // kappa bit 1: times -1
        re = -re;
        im = -im;
    }
    return make_float2(amp * re, amp * im);
}

// ---------------------------------------------------------------------------
// Operand image of the tensor-core contractions, one frequency: per tile of
// RB_TP pixels and plane (bf16 hi, lo), 2n / 8 rows of 1024 bf16, row rc holding
// r' = 8 rc .. 8 rc + 7 (r' = 2r + {0: Re G_r, 1: -Im G_r}) of the tile's pixels as
// 16 core matrices of 8 pixels x 16 bytes:
//   element (rc, x, r') at rc * 1024 + (x / 8) * 64 + (x % 8) * 8 + r' % 8.
// The adjoint reads it K-major, the forward MN-major (rb_born_tc.cu).
// ---------------------------------------------------------------------------
constexpr int RB_TP = 128;

// x = hi + lo with hi = bf16(x), lo = bf16(x - hi): x to ~2^-17 relative.
__device__ __forceinline__ void bf16_split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t bf16_pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Pixel p's 16 bytes of image row rc (elements 4 rc .. 4 rc + 3) in both planes of a
// tile (tile_img: the tile's hi plane; its lo plane follows after rcn rows).
__device__ __forceinline__ void aimg_put4(__nv_bfloat16* tile_img, int rcn, int rc, int p, const float2 g[4]) {
    uint32_t ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat16 h0, l0, h1, l1;
        bf16_split(g[q].x, h0, l0);
        bf16_split(-g[q].y, h1, l1);
        ah[q] = bf16_pack2(h0, h1);
        al[q] = bf16_pack2(l0, l1);
    }
    const size_t off = (size_t)(p >> 3) * 64 + (size_t)(p & 7) * 8;
    *(uint4*)(tile_img + (size_t)rc * 1024 + off) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
    *(uint4*)(tile_img + (size_t)(rcn + rc) * 1024 + off) = make_uint4(al[0], al[1], al[2], al[3]);
}

// Element t's position as float pairs.
__device__ __forceinline__ void elem_pos(const GeoDev& G, int t, DF& ex, DF& ey) {
    const float4 e = G.elem_xy[t];
    ex = DF{e.x, e.y};
    ey = DF{e.z, e.w};
}

// |pixel - x_t| as a float pair.
__device__ __forceinline__ DF pixel_elem_dist(const GeoDev& G, int ix, int iy, DF ex, DF ey) {
    DF X = df_pixel_coord(ix, G.cxg, G.h_hi, G.h_lo);
    DF Y = df_pixel_coord(iy, G.cyg, G.h_hi, G.h_lo);
    DF dx = df_sub(X, ex), dy = df_sub(Y, ey);
    DF d2 = df_add(df_sqr(dx), df_sqr(dy));
    if (d2.hi <= 0.f) return DF{0.f, 0.f};
    return df_sqrt(d2);
}

// ---------------------------------------------------------------------------
// Workspace layout (host side).
// ---------------------------------------------------------------------------
struct WsLayout {
    size_t elem_xy;    // [n_elem] float4 {x_hi, x_lo, y_hi, y_lo}
    size_t cells;      // [(ny-1)(nx-1)][8] float4
    size_t tables;     // [n_elem][npix] rb_cell
    size_t verts;      // [n_elem][max_steps + 1][n_rays] ray vertices, 32 B each (gridding)
    size_t gkeys;      // [n_elem][npix] u64 first-arrival keys (gridding)
    size_t ends;       // [n_elem][n_rays] rb_ray_end
    size_t fanlen;     // [n_elem] u32: vertices of each fan's longest ray (gridding)
    size_t counters;   // 64 uint32 + 64 double scalars
    size_t pray;       // [n_freq][n_elem][n_elem] float2 (ray data, then residual)
    size_t linked;     // [n_elem][n_elem] u8
    size_t wts;        // [n_freq][n_elem][n_elem] u8
    size_t keys;       // [n_freq][n_elem][n_elem] u64
    size_t sel;        // outlier selection scratch (rb_sel_bytes)
    size_t gsum;       // [npix] float
    size_t hsum;       // [npix] float
    size_t pdir;       // [npix] float
    size_t part;       // reduction partials: [n_part] double
    size_t fwd;        // forward partial sums: [n_chunks][n_elem][n_elem] float2
    size_t tcimg;      // tensor-core path: bf16 B-operand images, [n_freq][image]
    size_t gscr;       // tensor-core path: exact G per persistent CTA, [RB_TC_MAX_CTAS][n_elem][128] float2,
                       // the |G|^2 slices, then (Re g, H) per frequency [n_freq][npix] float2
    size_t tcfwd;      // tensor-core path: partial D blocks of the forward
    size_t aimg;       // tensor-core path: A operand images of the adjoint, [n_freq][...] bf16
    size_t cgv;        // CG variant: x, r, p, q vectors, [4][npix] float
    size_t tof;        // time-of-flight guess: link records, ray lengths and coefficients, pixel sums
    size_t total;
};

#define RB_TC_MAX_CTAS 160
size_t rb_ws_layout(const rb_geometry* g, int n_freq, rb_precision prec, WsLayout* L);
GeoDev rb_make_geo(const rb_geometry* g, const float4* elem_xy);
FreqC rb_make_freq(const rb_geometry* g, double f_hz);

// counters (uint32 slots)
enum { CNT_LOST = 0, CNT_HOLES = 1, CNT_UNLINKED = 2, CNT_KEPT = 3, CNT_ZEROED = 4, CNT_TC_TIMEOUT = 6, CNT_N = 64 };
// double scalars after the uint32 block
enum { DBL_EPS = 0, DBL_NUM = 1, DBL_DEN = 2, DBL_ALPHA = 3, DBL_NORM2 = 4, DBL_HMEAN = 5, DBL_N = 64 };
// CG variant: rho_k = <r_k, M^-1 r_k> at DBL_CG_RHO + k (k = 0..RB_MAX_CG) and the curvature
// <p_k, A p_k> at DBL_CG_PAP + k (k = 0..RB_MAX_CG-1)
enum { DBL_CG_RHO = 8, DBL_CG_PAP = DBL_CG_RHO + RB_MAX_CG + 1 };
static_assert(DBL_CG_PAP + RB_MAX_CG <= DBL_N, "CG scalars exceed the double block");

// One ray vertex in the vertex stream (written by the ray tracer when a buffer is
// given): position as float pairs, traveltime, q, l and the KMAH count (32 bytes).
struct Vtx { float xh, xl, yh, yl, t, q, l; int k; };

// Vertex k of ray i of fan t in the vertex stream: [fan][step][ray].
__device__ __forceinline__ size_t vtx_index(const GeoDev& G, int t, int k, int i) {
    return ((size_t)t * (size_t)(G.max_steps + 1) + (size_t)k) * (size_t)G.n_rays + (size_t)i;
}

// First-arrival link of one (emitter, receiver) pair: the traveltime, the winning
// interval (rays i, i + 1; -1 if unlinked) and the interpolation weight of ray i + 1.
struct LinkRec {
    double T;
    int32_t i;
    float lam;
};

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files); all return cudaGetLastError().
// ---------------------------------------------------------------------------
cudaError_t launch_elem_positions(const GeoDev& G, float4* elem_xy, cudaStream_t s);
cudaError_t launch_fields(const GeoDev& G, const float* c, const float* alpha0, float4* cells, cudaStream_t s);
// Rays; with keys set also the gridding: keys are reset here, and the tables (or, with
// images, the operand images) are written for every (element, pixel).
// traced (nullable): recorded on s once the rays' end records are written, before the
// rasteriser and the resolve pass.  keys_ready (nullable): the caller resets the keys
// (all ones) on another stream and records this event; s waits for it before the
// rasteriser instead of resetting them itself
// images (nullable, with F): the mixed path's operand images of every frequency of F,
// written by the resolve pass itself (tables then unused).  raster_mode: 0 the rule
// (along the tubes from 4 pixels per tube at the ring), 1 along the tubes, 2 across.
cudaError_t launch_trace(const GeoDev& G, const float4* cells, rb_ray_end* ends, const rb_rays* samples,
                         void* keys, rb_cell* tables, void* verts, const float* c, uint32_t* counters,
                         cudaStream_t s, cudaEvent_t traced = nullptr, cudaEvent_t keys_ready = nullptr,
                         const FreqSet* F = nullptr, void* images = nullptr, int raster_mode = 0,
                         uint32_t* fan_len = nullptr);
// Resets the first-arrival keys (n_elem * npix u64) to all ones, on s, with a fill
// narrow enough to run beside the tracer (for the keys_ready form of launch_trace).
cudaError_t launch_keys_reset(const GeoDev& G, void* keys, cudaStream_t s);
size_t rb_verts_bytes(int n_elem, int n_rays, int max_steps);
cudaError_t launch_green_out(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F,
                             float2* g_out, cudaStream_t s);
cudaError_t launch_link(const GeoDev& G, const float* c, const rb_ray_end* ends, const FreqSet& F,
                        float2* p_out, uint8_t* linked, cudaStream_t s, LinkRec* lrec = nullptr);
// outlier selection: histogram, scalars and candidates (rb_sel_bytes) in sel_ws
size_t rb_sel_bytes();
cudaError_t launch_residual_keys(const GeoDev& G, int n_freq, const float2* p_obs, float2* r_inout,
                                 const uint8_t* linked, uint64_t* keys, uint32_t* counters, void* sel_ws,
                                 cudaStream_t s);
cudaError_t launch_outlier_select(int n_total, double frac, const uint64_t* keys, uint32_t* counters, uint8_t* w,
                                  void* sel_ws, cudaStream_t s);
cudaError_t launch_adjoint_simt(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F,
                                const float2* resid, const uint8_t* w, float2* g_out, float* h_out,
                                float* gsum, float* hsum, uint32_t* counters, cudaStream_t s);
cudaError_t launch_forward_simt(const GeoDev& G, const rb_cell* tables, const float* c, const FreqC& F,
                                const float* m, float2* partial, int n_chunks, cudaStream_t s);
cudaError_t launch_forward_reduce(const GeoDev& G, const FreqC& F, const float2* partial, int n_chunks,
                                  float2* d_out, const uint8_t* w, double* den_part, cudaStream_t s);
int rb_fwd_chunks_for(int npix);
bool simt_adjoint_supported(int n_elem);
bool tc_adjoint_supported(int n_elem);
size_t tc_b_images_bytes(int n_elem);
cudaError_t launch_prep_b(int n, const float2* R, const uint8_t* W, void* img, cudaStream_t s);
size_t tc_forward_partial_bytes(int n_elem, int n_ctas);
cudaError_t launch_forward_tc(const GeoDev& G, const void* aimg, const FreqC& F, const float* m, float* partial,
                              int n_ctas, float2* d_out, const uint8_t* w, double* den_part, uint32_t* counters,
                              cudaStream_t s);
// The same with the split sum on stream r: the forward kernel on s, then (through
// fwd_done) its reduce on r, which records red_done when done, so the next frequency's
// forward on s can run beside it (its partial buffer must be another one).
cudaError_t launch_forward_tc_overlap(const GeoDev& G, const void* aimg, const FreqC& F, const float* m,
                                      float* partial, int n_ctas, float2* d_out, const uint8_t* w, double* den_part,
                                      uint32_t* counters, cudaStream_t s, cudaStream_t r, cudaEvent_t fwd_done,
                                      cudaEvent_t red_done);
// A images of the adjoint (and optionally the forward's G images) from the synthesis records
size_t tc_aimage_elems(int n_elem, int npix);
// operand images of F from the caller's tables (the single-operator entry points)
cudaError_t launch_tables_images(const GeoDev& G, const rb_cell* tables, const float* c, const FreqSet& F, void* aimg,
                                 cudaStream_t s);
cudaError_t launch_adjoint_tc(const GeoDev& G, const void* aimg, const FreqSet& F, const void* images, float2* gscr,
                              int n_ctas, float2* g_out, float* h_out, float* gsum, float* hsum, uint32_t* counters,
                              cudaStream_t s, int variant = 0);
cudaError_t launch_cg_init(const GeoDev& G, const float* gsum, const float* hsum, int precond, float* x, float* r,
                           float* p, double* part, double* dbl, double eps_rel, cudaStream_t s);
cudaError_t launch_cg_step(const GeoDev& G, const float* hsum, int precond, int k, float* x, float* r, float* p,
                           const float* q, double* part, double* dbl, cudaStream_t s);
size_t tof_ws_bytes(int n_elem, int n_rays, int npix);
cudaError_t launch_tof_link(const GeoDev& G, const float* c, const rb_ray_end* ends, void* tof_ws, uint8_t* linked,
                            cudaStream_t s);
cudaError_t launch_tof_times_out(const GeoDev& G, void* tof_ws, double* t_out, cudaStream_t s);
cudaError_t launch_tof_resid(const GeoDev& G, void* tof_ws, const double* t_obs, const uint8_t* obs_linked,
                             double* part, double* out, cudaStream_t s);
cudaError_t launch_tof_step(const GeoDev& G, const Vtx* verts, const rb_ray_end* ends, void* tof_ws, const double* t_obs,
                            const uint8_t* obs_linked, float* c, cudaStream_t s);
cudaError_t launch_cg_history(const double* dbl, int iters, double* hist, cudaStream_t s);
cudaError_t launch_sum_partials(const double* part, int n, double* dbl, int slot, double scale, int accumulate,
                                cudaStream_t s);
// limit_word (nullable, host-mapped): set to the lost-ray count when the update lost rays
cudaError_t launch_update(const GeoDev& G, float* c, const float* gsum, const float* hsum, float* pdir,
                          float* dc_out, double* part, double* dbl, uint32_t* counters, rb_diag* diag,
                          double eps_rel, int step_mode, int phase, cudaStream_t s, uint32_t* limit_word = nullptr);
