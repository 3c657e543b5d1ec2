// C-ABI entry points of librb: argument checks, workspace carving, launch order.
#include <math.h>
#include <string.h>

#include <mutex>

#include "rb_internal.cuh"

namespace {

constexpr double K_A = 11.512925464970229;  // 100 ln(10) / 20: dB/cm -> Np/m

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool geom_ok(const rb_geometry* g) {
    if (!g) return false;
    if (g->n_elem < 2 || g->n_elem > 1024) return false;
    if (g->nx < 3 || g->ny < 3 || g->nx > 4096 || g->ny > 4096) return false;
    if (!(g->h > 0.0) || !(g->ring_radius > 0.0) || !(g->ds > 0.0)) return false;
    if (g->n_rays < 2 || g->n_rays > 4096) return false;
    if (g->max_steps < 1 || g->max_steps > (1 << 20)) return false;
    if (!(g->support_margin >= 0.0) || !(g->support_margin < g->ring_radius)) return false;
    if (!(g->c_ref > 0.0) || !(g->f_ref > 0.0) || !(g->power_y > 0.0) || !(g->power_y < 3.0)) return false;
    // the ring must lie inside the grid
    const double half = 0.5 * (double)((g->nx < g->ny ? g->nx : g->ny) - 1) * g->h;
    if (!(g->ring_radius < half)) return false;
    // triangle ids must fit the 24-bit field of the table tag
    const double ids = 2.0 * (double)(g->n_rays - 1) * (double)(g->max_steps + 1);
    if (ids >= 16777216.0) return false;
    return true;
}

GeoDev make_geo(const rb_geometry* g, const float4* elem_xy) {
    GeoDev G;
    G.n_elem = g->n_elem;
    G.nx = g->nx;
    G.ny = g->ny;
    G.fxmax = (float)(g->nx - 1);
    G.fymax = (float)(g->ny - 1);
    G.n_rays = g->n_rays;
    G.max_steps = g->max_steps;
    G.npix = g->nx * g->ny;
    G.h = (float)g->h;
    G.inv_h = (float)(1.0 / g->h);
    G.cxg = 0.5f * (float)(g->nx - 1);
    G.cyg = 0.5f * (float)(g->ny - 1);
    const DF hd = df_from_double(g->h);
    G.h_hi = hd.hi;
    G.h_lo = hd.lo;
    G.ds = (float)g->ds;
    G.R = (float)g->ring_radius;
    G.R2 = (float)(g->ring_radius * g->ring_radius);
    G.inv_cref = (float)(1.0 / g->c_ref);
    G.inv_cref_lo = (float)(1.0 / g->c_ref - (double)G.inv_cref);
    G.c_ref = (float)g->c_ref;
    G.j_floor = (float)(0.25 * g->h);
    G.R_d = g->ring_radius;
    G.ds_d = g->ds;
    G.c_ref_d = g->c_ref;
    G.h_d = g->h;
    const double q = 2.0 * (g->ring_radius - g->support_margin) / g->h;
    G.r2max = (long long)floor(q * q);
    G.elem_xy = elem_xy;
    return G;
}

// dispersion phase per unit alpha0 integral [rad]: causal power law relative to f_ref
double dispersion_phase(double f, double y, double f_ref) {
    const double w = 2.0 * M_PI * f, wr = 2.0 * M_PI * f_ref;
    if (y == 1.0) return -(2.0 / M_PI) * w * log(w / wr) * K_A / (2.0 * M_PI * 1e6);
    const double diff = pow(wr, y - 1.0) * expm1((y - 1.0) * log(w / wr));
    return w * tan(0.5 * M_PI * y) * diff * K_A * pow(2.0 * M_PI * 1e6, -y);
}

FreqC make_freq(const rb_geometry* g, double f) {
    FreqC F;
    const double w = 2.0 * M_PI * f;
    F.f_d = f;
    F.f_hi = (float)f;
    F.f_lo = (float)(f - (double)F.f_hi);
    const DF kf = df_from_double(f / g->c_ref);
    F.kf_hi = kf.hi;
    F.kf_lo = kf.lo;
    F.w_isqrt = (float)(1.0 / sqrt(w));
    F.a_abs = (float)(K_A * pow(f / 1e6, g->power_y));
    F.disp_cyc = (float)(dispersion_phase(f, g->power_y, g->f_ref) / (2.0 * M_PI));
    F.w2 = (float)(w * w);
    F.w4 = (float)(w * w * w * w);
    return F;
}

bool make_freqs(const rb_geometry* g, const double* f, int n, FreqSet* F) {
    if (!f || n < 1 || n > RB_MAX_FREQ) return false;
    F->n = n;
    for (int i = 0; i < n; ++i) {
        if (!(f[i] > 0.0) || !isfinite(f[i])) return false;
        F->f[i] = make_freq(g, f[i]);
    }
    return true;
}

struct Ws {
    WsLayout L;
    char* base;
    template <class T> T* at(size_t off) const { return (T*)(base + off); }
};

rb_status check_ws(const rb_geometry* g, int n_freq, rb_precision prec, void* ws, size_t ws_bytes, Ws* W) {
    if (!ws) return RB_ERR_WORKSPACE;
    if (((uintptr_t)ws & 255) != 0) return RB_ERR_WORKSPACE;
    const size_t need = rb_ws_layout(g, n_freq, prec, &W->L);
    if (need == 0) return RB_ERR_SHAPE;
    if (ws_bytes < need) return RB_ERR_WORKSPACE;
    W->base = (char*)ws;
    return RB_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int tc_ctas() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    return n < RB_TC_MAX_CTAS ? n : RB_TC_MAX_CTAS;
}

#define RB_CU(x)                                   \
    do {                                           \
        if ((x) != cudaSuccess) return RB_ERR_CUDA; \
    } while (0)

// A side stream per (device, caller stream) for the work of an update that need not sit
// on the caller's stream: the first-arrival keys reset beside the ray trace, the work
// that does not wait for the gridding (linking, residuals, data weights, B images),
// forked after the trace and joined before the adjoint, and each frequency's forward
// reduce beside the next forward; so that updates issued on different streams (the
// requests of a server) do not queue behind one another's side work.  Created on first
// use and kept for the process (at most kMaxSide; beyond that, callers share the entries
// of their device, which stays correct and only serialises their side work); the mutex
// keeps each call's fork and join events together when several host threads call.
// With each entry goes a word of host-mapped memory: the update that loses rays writes
// its lost-ray count there from the device, and the next update call from the same
// stream with the same workspace that finds it set clears it and returns RB_ERR_LIMIT
// without launching anything (no synchronisation: the word is seen once the lossy update
// has completed).  A call with another workspace (a new problem on a reused stream)
// discards a pending report that belonged to the previous one.
struct SideStream {
    int dev = -1;
    cudaStream_t caller = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t start = nullptr, keys = nullptr, fork = nullptr, join = nullptr;
    cudaEvent_t fwd[2] = {nullptr, nullptr}, red[2] = {nullptr, nullptr};   // forward / its reduce, by parity
    uint32_t* lim_host = nullptr;   // null when host-mapped memory is unavailable
    uint32_t* lim_dev = nullptr;
    const void* last_ws = nullptr;  // workspace of the stream's last update
};
constexpr int kMaxSide = 256;
constexpr int kLimitStride = 16;   // one 64-byte line per entry
std::mutex g_side_mutex;
SideStream g_side[kMaxSide];
int g_side_n = 0;
alignas(4096) uint32_t g_limit_words[kMaxSide * kLimitStride];
int g_limit_state = 0;   // 0: not registered yet, 1: registered (mapped, portable), -1: unavailable

// The device address of limit word k on the current device (null if unavailable).
uint32_t* limit_word_dev(int k) {
    if (g_limit_state == 0) {
        g_limit_state = cudaHostRegister(g_limit_words, sizeof(g_limit_words),
                                         cudaHostRegisterMapped | cudaHostRegisterPortable) == cudaSuccess ? 1 : -1;
        if (g_limit_state < 0) cudaGetLastError();
    }
    if (g_limit_state < 0) return nullptr;
    void* p = nullptr;
    if (cudaHostGetDevicePointer(&p, g_limit_words, 0) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    return (uint32_t*)p + (size_t)k * kLimitStride;
}

cudaError_t side_stream(cudaStream_t caller, SideStream** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int any = -1;
    for (int k = 0; k < g_side_n; ++k) {
        if (g_side[k].dev != dev) continue;
        if (g_side[k].caller == caller) {
            *out = &g_side[k];
            return cudaSuccess;
        }
        if (any < 0) any = k;
    }
    if (g_side_n == kMaxSide) {
        if (any < 0) return cudaErrorInvalidDevice;
        *out = &g_side[any];   // table full: share an entry of this device
        return cudaSuccess;
    }
    // built aside and published whole, so a failed creation leaves no half-made entry;
    // the first call may come inside a stream capture, so this thread's capture mode is
    // relaxed around the creation and restored after it
    SideStream n;
    n.dev = dev;
    n.caller = caller;
    cudaEvent_t* evs[8] = {&n.start, &n.keys, &n.fork, &n.join, &n.fwd[0], &n.fwd[1], &n.red[0], &n.red[1]};
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    if ((e = cudaThreadExchangeStreamCaptureMode(&mode)) != cudaSuccess) return e;
    e = cudaStreamCreateWithFlags(&n.s, cudaStreamNonBlocking);
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(evs[k], cudaEventDisableTiming);
    if (e == cudaSuccess) {
        n.lim_dev = limit_word_dev(g_side_n);
        if (n.lim_dev) {
            n.lim_host = g_limit_words + (size_t)g_side_n * kLimitStride;
            __atomic_store_n(n.lim_host, 0u, __ATOMIC_RELEASE);
        }
    }
    cudaThreadExchangeStreamCaptureMode(&mode);
    if (e != cudaSuccess) {
        for (int k = 0; k < 8; ++k)
            if (*evs[k]) cudaEventDestroy(*evs[k]);
        if (n.s) cudaStreamDestroy(n.s);
        return e;
    }
    g_side[g_side_n] = n;
    *out = &g_side[g_side_n++];
    return cudaSuccess;
}

// Stage events of the update entry points (none when the caller gave no array).
struct Marks {
    cudaEvent_t* ev;
    cudaStream_t s;
    cudaError_t operator()(int stage, int end) const { return ev ? cudaEventRecord(ev[2 * stage + end], s) : cudaSuccess; }
};

rb_status check_update(const rb_geometry* geom, const float* c, const float* alpha0, const double* freqs_hz,
                       int n_freq, const float* p_obs, const rb_update_params* params, rb_precision prec,
                       FreqSet* F) {
    if (!geom || !c || !alpha0 || !p_obs || !params) return RB_ERR_ARG;
    if (prec != RB_PREC_FP32 && prec != RB_PREC_BF16X3) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    if (!(params->outlier_frac >= 0.0 && params->outlier_frac < 1.0)) return RB_ERR_ARG;
    if (!(params->eps_rel >= 0.0) || !isfinite(params->eps_rel)) return RB_ERR_ARG;
    if (params->step_mode != RB_STEP_EXACT && params->step_mode != RB_STEP_DIAG) return RB_ERR_ARG;
    if ((params->tune & ~15) != 0 || (params->tune & 3) == 3 || ((params->tune >> 2) & 3) == 3) return RB_ERR_ARG;
    if (!make_freqs(geom, freqs_hz, n_freq, F)) return RB_ERR_ARG;
    if (prec == RB_PREC_BF16X3 && !tc_adjoint_supported(geom->n_elem)) return RB_ERR_UNSUPPORTED;
    if (prec == RB_PREC_FP32 && !simt_adjoint_supported(geom->n_elem)) return RB_ERR_UNSUPPORTED;
    return RB_OK;
}

// The stages both updates share (Secs. 3-4): fields, rays and first-arrival tables,
// linking, residuals and data weights, the operand images (mixed path), and the
// gradient sum_w Re g_w -> gsum and Hessian diagonal sum_w H_w -> hsum.
rb_status gradient_stages(const GeoDev& G, const FreqSet& F, const Ws& W, float* c, const float* alpha0,
                          const float* p_obs, const rb_update_params* params, rb_precision prec, const Marks& mark,
                          cudaStream_t s, uint32_t** limit_word) {
    const int n_freq = F.n;
    const int ne2 = G.n_elem * G.n_elem;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    float4* cells = W.at<float4>(W.L.cells);
    rb_cell* tables = W.at<rb_cell>(W.L.tables);
    rb_ray_end* ends = W.at<rb_ray_end>(W.L.ends);
    float2* R = W.at<float2>(W.L.pray);
    uint8_t* linked = W.at<uint8_t>(W.L.linked);
    uint8_t* wts = W.at<uint8_t>(W.L.wts);
    uint64_t* keys = W.at<uint64_t>(W.L.keys);
    const bool tc = prec == RB_PREC_BF16X3;
    std::lock_guard<std::mutex> lock(g_side_mutex);
    SideStream* ss = nullptr;
    RB_CU(side_stream(s, &ss));
    // an earlier update from this stream and workspace lost rays: report it once, launching nothing
    if (ss->lim_host) {
        const bool same = ss->last_ws == (const void*)W.base;
        ss->last_ws = (const void*)W.base;
        if (__atomic_exchange_n(ss->lim_host, 0u, __ATOMIC_ACQ_REL) != 0 && same) return RB_ERR_LIMIT;
    }
    *limit_word = ss->lim_dev;
    const cudaStream_t s2 = ss->s;
    const Marks mark2{mark.ev, s2};   // stage events of the side branch
    RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4 + DBL_N * 8, s));
    RB_CU(mark(RB_STAGE_FIELDS, 0));
    RB_CU(launch_elem_positions(G, exy, s));
    RB_CU(launch_fields(G, c, alpha0, cells, s));
    // side branch 1: the first-arrival keys reset (all ones) beside the tracer; forked
    // after the fields, which it would otherwise slow (0.098 against 0.031 ms on a
    // 256-element ring at 512^2 pixels), by a fill of one CTA per SM
    RB_CU(cudaEventRecord(ss->start, s));
    RB_CU(cudaStreamWaitEvent(s2, ss->start, 0));
    RB_CU(launch_keys_reset(G, W.at<void>(W.L.gkeys), s2));
    RB_CU(cudaEventRecord(ss->keys, s2));
    RB_CU(mark(RB_STAGE_FIELDS, 1));
    RB_CU(mark(RB_STAGE_TRACE_GRID, 0));
    // the plain path reads the tables; on the mixed path the resolve pass writes the
    // operand images of the set itself
    RB_CU(launch_trace(G, cells, ends, nullptr, W.at<void>(W.L.gkeys), tc ? nullptr : tables, W.at<void>(W.L.verts), c,
                       cnt, s, ss->fork, ss->keys, tc ? &F : nullptr, tc ? W.at<void>(W.L.aimg) : nullptr,
                       params->tune & 3, W.at<uint32_t>(W.L.fanlen)));
    // side branch 2 (needs the end records only): links, residuals, weights, B images
    RB_CU(cudaStreamWaitEvent(s2, ss->fork, 0));
    RB_CU(mark2(RB_STAGE_LINK, 0));
    RB_CU(launch_link(G, c, ends, F, R, linked, s2));
    RB_CU(launch_residual_keys(G, n_freq, (const float2*)p_obs, R, linked, keys, cnt, W.at<void>(W.L.sel), s2));
    RB_CU(launch_outlier_select(n_freq * ne2, params->outlier_frac, keys, cnt, wts, W.at<void>(W.L.sel), s2));
    if (tc) {
        const size_t img = tc_b_images_bytes(G.n_elem);
        for (int w = 0; w < n_freq; ++w)
            RB_CU(launch_prep_b(G.n_elem, R + (size_t)w * ne2, wts + (size_t)w * ne2, W.at<char>(W.L.tcimg) + w * img,
                                s2));
    }
    RB_CU(mark2(RB_STAGE_LINK, 1));
    RB_CU(cudaEventRecord(ss->join, s2));
    // main branch: rasteriser and resolve (in launch_trace; on the mixed path with the
    // operand images, so the images stage is empty)
    RB_CU(mark(RB_STAGE_TRACE_GRID, 1));
    RB_CU(mark(RB_STAGE_IMAGES, 0));
    RB_CU(mark(RB_STAGE_IMAGES, 1));
    RB_CU(cudaStreamWaitEvent(s, ss->join, 0));
    RB_CU(mark(RB_STAGE_ADJOINT, 0));
    if (tc) {
        RB_CU(launch_adjoint_tc(G, W.at<void>(W.L.aimg), F, W.at<void>(W.L.tcimg), W.at<float2>(W.L.gscr), tc_ctas(),
                                nullptr, nullptr, W.at<float>(W.L.gsum), W.at<float>(W.L.hsum), cnt, s,
                                (params->tune >> 2) & 3));
    } else {
        RB_CU(launch_adjoint_simt(G, tables, c, F, R, wts, nullptr, nullptr, W.at<float>(W.L.gsum),
                                  W.at<float>(W.L.hsum), cnt, s));
    }
    RB_CU(mark(RB_STAGE_ADJOINT, 1));
    return RB_OK;
}

}  // namespace

GeoDev rb_make_geo(const rb_geometry* g, const float4* elem_xy) { return make_geo(g, elem_xy); }
FreqC rb_make_freq(const rb_geometry* g, double f_hz) { return make_freq(g, f_hz); }

size_t rb_ws_layout(const rb_geometry* g, int n_freq, rb_precision prec, WsLayout* L) {
    if (!geom_ok(g) || n_freq < 1 || n_freq > RB_MAX_FREQ) return 0;
    const bool tcp = prec == RB_PREC_BF16X3;
    const size_t ne = (size_t)g->n_elem, npix = (size_t)g->nx * g->ny;
    const size_t ncell = (size_t)(g->nx - 1) * (g->ny - 1);
    const size_t nf = (size_t)n_freq;
    size_t o = 0;
    L->counters = o; o = align256(o + CNT_N * 4 + DBL_N * 8);
    L->elem_xy = o; o = align256(o + ne * 16);
    L->cells = o; o = align256(o + ncell * 128);
    // the plain path's tables and forward partials; the mixed path keeps neither (its
    // resolve pass writes the operand images)
    L->tables = o; o = align256(o + (tcp ? 0 : ne * npix * sizeof(rb_cell)));
    L->verts = o; o = align256(o + rb_verts_bytes(g->n_elem, g->n_rays, g->max_steps));
    L->gkeys = o; o = align256(o + ne * npix * 8);
    L->ends = o; o = align256(o + ne * (size_t)g->n_rays * sizeof(rb_ray_end));
    L->fanlen = o; o = align256(o + ne * 4);
    L->pray = o; o = align256(o + nf * ne * ne * 8);
    L->linked = o; o = align256(o + ne * ne);
    L->wts = o; o = align256(o + nf * ne * ne);
    L->keys = o; o = align256(o + nf * ne * ne * 8);
    L->sel = o; o = align256(o + rb_sel_bytes());
    L->gsum = o; o = align256(o + npix * 4);
    L->hsum = o; o = align256(o + npix * 4);
    L->pdir = o; o = align256(o + npix * 4);
    L->part = o; o = align256(o + (size_t)(RB_MAX_FREQ + 2) * 256 * 8);
    L->fwd = o; o = align256(o + (tcp ? 0 : (size_t)rb_fwd_chunks_for((int)npix) * ne * ne * 8));
    L->tcimg = o; o = align256(o + (tcp ? (size_t)n_freq * tc_b_images_bytes(g->n_elem) : 0));
    // exact G per persistent CTA, then its |G|^2 A slices (bf16 hi and lo), then (Re g, H)
    // of each frequency of the set for the adjoint's sums over the set
    L->gscr = o; o = align256(o + (tcp ? (size_t)RB_TC_MAX_CTAS * ne * 128 * (8 + 4) + nf * npix * 8 : 0));
    // two of them on the update path: one frequency's reduce runs beside the next one's forward
    L->tcfwd = o; o = align256(o + (tcp ? 2 * align256(tc_forward_partial_bytes(g->n_elem, RB_TC_MAX_CTAS)) : 0));
    L->aimg = o; o = align256(o + (tcp ? (size_t)n_freq * tc_aimage_elems(g->n_elem, (int)npix) * 2 : 0));
    L->cgv = o; o = align256(o + 4 * npix * 4);
    L->tof = o; o = align256(o + tof_ws_bytes(g->n_elem, g->n_rays, (int)npix));
    // one size fits every entry point: the single-precision calls (rays, gridding, data
    // weights, times of flight) lay the same workspace out as the FP32 path does
    if (tcp) {
        WsLayout L32;
        const size_t o32 = rb_ws_layout(g, n_freq, RB_PREC_FP32, &L32);
        if (o32 > o) o = o32;
    }
    L->total = o;
    return o;
}

extern "C" {

size_t rb_workspace_size(const rb_geometry* geom, int32_t n_freq, rb_precision prec) {
    WsLayout L;
    if (prec != RB_PREC_FP32 && prec != RB_PREC_BF16X3) return 0;
    return rb_ws_layout(geom, n_freq, prec, &L);
}

const char* rb_status_string(rb_status s) {
    switch (s) {
        case RB_OK: return "ok";
        case RB_ERR_ARG: return "invalid argument";
        case RB_ERR_SHAPE: return "unsupported sizes";
        case RB_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case RB_ERR_CUDA: return "CUDA launch or call failed";
        case RB_ERR_LIMIT: return "device-side limit reached";
        case RB_ERR_UNSUPPORTED: return "not supported by the library";
    }
    return "unknown status";
}

rb_status rb_trace_rays(const rb_geometry* geom, const float* c, const float* alpha0, rb_rays* out, void* ws,
                        size_t ws_bytes, rb_stream stream) {
    if (!geom || !c || !alpha0 || !out || !out->ends) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    const bool any = out->vx || out->vy || out->vt || out->vq || out->vl || out->vkappa;
    const bool all = out->vx && out->vy && out->vt && out->vq && out->vl && out->vkappa;
    if (any && !all) return RB_ERR_ARG;
    Ws W;
    rb_status st = check_ws(geom, 1, RB_PREC_FP32, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
    RB_CU(launch_elem_positions(G, exy, s));
    RB_CU(launch_fields(G, c, alpha0, W.at<float4>(W.L.cells), s));
    RB_CU(launch_trace(G, W.at<float4>(W.L.cells), out->ends, out, nullptr, nullptr, nullptr, nullptr, cnt, s));
    return RB_OK;
}

rb_status rb_green_grid(const rb_geometry* geom, const float* c, const float* alpha0, rb_cell* tables,
                        const double* freqs_hz, int32_t n_freq, float* g_out, void* ws, size_t ws_bytes,
                        rb_stream stream) {
    if (!geom || !c || !alpha0 || !tables) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    if (!aligned16(tables)) return RB_ERR_ARG;
    FreqSet F;
    F.n = 0;
    if (g_out && !make_freqs(geom, freqs_hz, n_freq, &F)) return RB_ERR_ARG;
    Ws W;
    rb_status st = check_ws(geom, 1, RB_PREC_FP32, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
    RB_CU(launch_elem_positions(G, exy, s));
    RB_CU(launch_fields(G, c, alpha0, W.at<float4>(W.L.cells), s));
    RB_CU(launch_trace(G, W.at<float4>(W.L.cells), W.at<rb_ray_end>(W.L.ends), nullptr, W.at<void>(W.L.gkeys), tables,
                       W.at<void>(W.L.verts), nullptr, cnt, s, nullptr, nullptr, nullptr, nullptr, 0,
                       W.at<uint32_t>(W.L.fanlen)));
    if (g_out) RB_CU(launch_green_out(G, tables, c, F, (float2*)g_out, s));
    return RB_OK;
}

rb_status rb_ray_forward(const rb_geometry* geom, const float* c, const rb_ray_end* ends, const double* freqs_hz,
                         int32_t n_freq, float* p_out, uint8_t* linked_out, rb_stream stream) {
    if (!geom || !c || !ends || !p_out) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    FreqSet F;
    if (!make_freqs(geom, freqs_hz, n_freq, &F)) return RB_ERR_ARG;
    const GeoDev G = make_geo(geom, nullptr);
    RB_CU(launch_link(G, c, ends, F, (float2*)p_out, linked_out, (cudaStream_t)stream));
    return RB_OK;
}

rb_status rb_data_weights(const rb_geometry* geom, const float* c, const float* alpha0, const double* freqs_hz,
                          int32_t n_freq, const float* p_obs, double outlier_frac, float* resid_out, uint8_t* w_out,
                          void* ws, size_t ws_bytes, rb_stream stream) {
    if (!geom || !c || !alpha0 || !p_obs || !resid_out || !w_out) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    if (!(outlier_frac >= 0.0 && outlier_frac < 1.0)) return RB_ERR_ARG;
    FreqSet F;
    if (!make_freqs(geom, freqs_hz, n_freq, &F)) return RB_ERR_ARG;
    Ws W;
    rb_status st = check_ws(geom, n_freq, RB_PREC_FP32, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    rb_ray_end* ends = W.at<rb_ray_end>(W.L.ends);
    uint8_t* linked = W.at<uint8_t>(W.L.linked);
    float2* R = (float2*)resid_out;
    RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
    RB_CU(launch_elem_positions(G, exy, s));
    RB_CU(launch_fields(G, c, alpha0, W.at<float4>(W.L.cells), s));
    RB_CU(launch_trace(G, W.at<float4>(W.L.cells), ends, nullptr, nullptr, nullptr, nullptr, nullptr, cnt, s));
    RB_CU(launch_link(G, c, ends, F, R, linked, s));
    RB_CU(launch_residual_keys(G, n_freq, (const float2*)p_obs, R, linked, W.at<uint64_t>(W.L.keys), cnt,
                               W.at<void>(W.L.sel), s));
    RB_CU(launch_outlier_select(n_freq * G.n_elem * G.n_elem, outlier_frac, W.at<uint64_t>(W.L.keys), cnt, w_out,
                                W.at<void>(W.L.sel), s));
    return RB_OK;
}

rb_status rb_born_forward(const rb_geometry* geom, const rb_cell* tables, const float* c, double f_hz, const float* m,
                          float* d_out, rb_precision prec, void* ws, size_t ws_bytes, rb_stream stream) {
    if (!geom || !tables || !c || !m || !d_out) return RB_ERR_ARG;
    if (prec != RB_PREC_FP32 && prec != RB_PREC_BF16X3) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    if (!(f_hz > 0.0) || !isfinite(f_hz)) return RB_ERR_ARG;
    if (prec == RB_PREC_BF16X3 && !tc_adjoint_supported(geom->n_elem)) return RB_ERR_UNSUPPORTED;
    Ws W;
    rb_status st = check_ws(geom, 1, prec, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    const FreqC F = make_freq(geom, f_hz);
    const int nch = rb_fwd_chunks_for(G.npix);
    RB_CU(launch_elem_positions(G, exy, s));
    if (prec == RB_PREC_BF16X3) {
        RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
        FreqSet F1;
        F1.n = 1;
        F1.f[0] = F;
        RB_CU(launch_tables_images(G, tables, c, F1, W.at<void>(W.L.aimg), s));
        RB_CU(launch_forward_tc(G, W.at<void>(W.L.aimg), F, m, W.at<float>(W.L.tcfwd), tc_ctas(), (float2*)d_out,
                                nullptr, nullptr, cnt, s));
    } else {
        RB_CU(launch_forward_simt(G, tables, c, F, m, W.at<float2>(W.L.fwd), nch, s));
        RB_CU(launch_forward_reduce(G, F, W.at<float2>(W.L.fwd), nch, (float2*)d_out, nullptr, nullptr, s));
    }
    return RB_OK;
}

rb_status rb_born_adjoint(const rb_geometry* geom, const rb_cell* tables, const float* c, double f_hz,
                          const float* resid, const uint8_t* w, float* g_out, float* hdiag_out, rb_precision prec,
                          void* ws, size_t ws_bytes, rb_stream stream) {
    if (!geom || !tables || !c || !resid || !w || !g_out) return RB_ERR_ARG;
    if (prec != RB_PREC_FP32 && prec != RB_PREC_BF16X3) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    if (!(f_hz > 0.0) || !isfinite(f_hz)) return RB_ERR_ARG;
    if (prec == RB_PREC_BF16X3 && !tc_adjoint_supported(geom->n_elem)) return RB_ERR_UNSUPPORTED;
    if (prec == RB_PREC_FP32 && !simt_adjoint_supported(geom->n_elem)) return RB_ERR_UNSUPPORTED;
    Ws W;
    rb_status st = check_ws(geom, 1, prec, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    FreqSet F;
    F.n = 1;
    F.f[0] = make_freq(geom, f_hz);
    RB_CU(launch_elem_positions(G, exy, s));
    if (prec == RB_PREC_BF16X3) {
        RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
        RB_CU(launch_prep_b(G.n_elem, (const float2*)resid, w, W.at<void>(W.L.tcimg), s));
        RB_CU(launch_tables_images(G, tables, c, F, W.at<void>(W.L.aimg), s));
        RB_CU(launch_adjoint_tc(G, W.at<void>(W.L.aimg), F, W.at<void>(W.L.tcimg), W.at<float2>(W.L.gscr), tc_ctas(),
                                (float2*)g_out, hdiag_out, nullptr, nullptr, cnt, s));
    } else {
        RB_CU(launch_adjoint_simt(G, tables, c, F, (const float2*)resid, w, (float2*)g_out, hdiag_out, nullptr,
                                  nullptr, nullptr, s));
    }
    return RB_OK;
}

rb_status rb_hf_update(const rb_geometry* geom, float* c_inout, const float* alpha0, const double* freqs_hz,
                       int32_t n_freq, const float* p_obs, const rb_update_params* params, rb_precision prec,
                       float* dc_out, rb_diag* diag_out, void* ws, size_t ws_bytes, rb_stream stream) {
    FreqSet F;
    rb_status st = check_update(geom, c_inout, alpha0, freqs_hz, n_freq, p_obs, params, prec, &F);
    if (st != RB_OK) return st;
    Ws W;
    st = check_ws(geom, n_freq, prec, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const GeoDev G = make_geo(geom, W.at<float4>(W.L.elem_xy));
    const Marks mark{(cudaEvent_t*)params->stage_events, s};
    uint32_t* limit_word = nullptr;
    st = gradient_stages(G, F, W, c_inout, alpha0, p_obs, params, prec, mark, s, &limit_word);
    if (st != RB_OK) return st;
    const int ne2 = G.n_elem * G.n_elem;
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    double* dbl = (double*)(cnt + CNT_N);
    rb_cell* tables = W.at<rb_cell>(W.L.tables);
    uint8_t* wts = W.at<uint8_t>(W.L.wts);
    float* gsum = W.at<float>(W.L.gsum);
    float* hsum = W.at<float>(W.L.hsum);
    float* pdir = W.at<float>(W.L.pdir);
    double* part = W.at<double>(W.L.part);
    float2* fwd = W.at<float2>(W.L.fwd);
    const int nch = rb_fwd_chunks_for(G.npix);
    RB_CU(mark(RB_STAGE_DIRECTION, 0));
    RB_CU(launch_update(G, c_inout, gsum, hsum, pdir, dc_out, part, dbl, cnt, diag_out, params->eps_rel,
                        params->step_mode, 0, s));
    RB_CU(mark(RB_STAGE_DIRECTION, 1));
    RB_CU(mark(RB_STAGE_FORWARD, 0));
    if (params->step_mode == RB_STEP_EXACT) {
        SideStream* ss = nullptr;
        if (prec == RB_PREC_BF16X3) {
            std::lock_guard<std::mutex> lock(g_side_mutex);
            RB_CU(side_stream(s, &ss));
        }
        const size_t half = align256(tc_forward_partial_bytes(G.n_elem, RB_TC_MAX_CTAS));
        for (int w = 0; w < n_freq; ++w) {
            if (prec == RB_PREC_BF16X3) {
                // frequency w's reduce runs on the side stream beside frequency w + 1's forward;
                // the forward of w + 2 reuses w's partial buffer once w's reduce is done
                if (w >= 2) RB_CU(cudaStreamWaitEvent(s, ss->red[w & 1], 0));
                RB_CU(launch_forward_tc_overlap(G, W.at<char>(W.L.aimg) + (size_t)w * tc_aimage_elems(G.n_elem, G.npix) * 2,
                                                F.f[w], pdir, (float*)(W.at<char>(W.L.tcfwd) + (w & 1) * half), tc_ctas(),
                                                nullptr, wts + (size_t)w * ne2, part + (size_t)w * 256, cnt, s, ss->s,
                                                ss->fwd[w & 1], ss->red[w & 1]));
                if (w == n_freq - 1) RB_CU(cudaStreamWaitEvent(s, ss->red[w & 1], 0));   // the last reduce (the
                                                                                          // others precede it)
            } else {
                RB_CU(launch_forward_simt(G, tables, c_inout, F.f[w], pdir, fwd, nch, s));
                RB_CU(launch_forward_reduce(G, F.f[w], fwd, nch, nullptr, wts + (size_t)w * ne2,
                                            part + (size_t)w * 256, s));
            }
        }
        RB_CU(launch_sum_partials(part, n_freq * 256, dbl, DBL_DEN, 1.0, 0, s));
    }
    RB_CU(mark(RB_STAGE_FORWARD, 1));
    RB_CU(mark(RB_STAGE_APPLY, 0));
    RB_CU(launch_update(G, c_inout, gsum, hsum, pdir, dc_out, part + (size_t)RB_MAX_FREQ * 256, dbl, cnt, diag_out,
                        params->eps_rel, params->step_mode, 1, s, limit_word));
    RB_CU(mark(RB_STAGE_APPLY, 1));
    return RB_OK;
}

rb_status rb_cg_update(const rb_geometry* geom, float* c_inout, const float* alpha0, const double* freqs_hz,
                       int32_t n_freq, const float* p_obs, const rb_update_params* params, int32_t cg_iters,
                       int32_t precond, rb_precision prec, float* dc_out, double* cg_hist_out, rb_diag* diag_out,
                       void* ws, size_t ws_bytes, rb_stream stream) {
    if (cg_iters < 1 || cg_iters > RB_MAX_CG || (precond != 0 && precond != 1)) return RB_ERR_ARG;
    FreqSet F;
    rb_status st = check_update(geom, c_inout, alpha0, freqs_hz, n_freq, p_obs, params, prec, &F);
    if (st != RB_OK) return st;
    Ws W;
    st = check_ws(geom, n_freq, prec, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const GeoDev G = make_geo(geom, W.at<float4>(W.L.elem_xy));
    const Marks mark{(cudaEvent_t*)params->stage_events, s};
    uint32_t* limit_word = nullptr;
    st = gradient_stages(G, F, W, c_inout, alpha0, p_obs, params, prec, mark, s, &limit_word);
    if (st != RB_OK) return st;
    const int ne2 = G.n_elem * G.n_elem;
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    double* dbl = (double*)(cnt + CNT_N);
    rb_cell* tables = W.at<rb_cell>(W.L.tables);
    uint8_t* wts = W.at<uint8_t>(W.L.wts);
    float* gsum = W.at<float>(W.L.gsum);
    float* hsum = W.at<float>(W.L.hsum);
    double* part = W.at<double>(W.L.part);
    double* vpart = part + (size_t)RB_MAX_FREQ * 256;
    float* x = W.at<float>(W.L.cgv);
    float* r = x + G.npix;
    float* p = r + G.npix;
    float* q = p + G.npix;
    // the residuals are consumed by the gradient: their buffer holds B_w p from here on
    float2* d = W.at<float2>(W.L.pray);
    const bool tc = prec == RB_PREC_BF16X3;
    const size_t img = tc_b_images_bytes(G.n_elem);
    const int nch = rb_fwd_chunks_for(G.npix);
    RB_CU(mark(RB_STAGE_DIRECTION, 0));
    RB_CU(launch_cg_init(G, gsum, hsum, precond, x, r, p, part, dbl, params->eps_rel, s));
    RB_CU(mark(RB_STAGE_DIRECTION, 1));
    RB_CU(mark(RB_STAGE_FORWARD, 0));
    for (int k = 0; k < cg_iters; ++k) {
        // B_w p for every frequency of the set, and sum_w sum W |B_w p|^2
        for (int w = 0; w < n_freq; ++w) {
            float2* dw = d + (size_t)w * ne2;
            if (tc) {
                RB_CU(launch_forward_tc(G, W.at<char>(W.L.aimg) + (size_t)w * tc_aimage_elems(G.n_elem, G.npix) * 2,
                                        F.f[w], p, W.at<float>(W.L.tcfwd), tc_ctas(), dw, wts + (size_t)w * ne2,
                                        part + (size_t)w * 256, cnt, s));
                RB_CU(launch_prep_b(G.n_elem, dw, wts + (size_t)w * ne2, W.at<char>(W.L.tcimg) + w * img, s));
            } else {
                RB_CU(launch_forward_simt(G, tables, c_inout, F.f[w], p, W.at<float2>(W.L.fwd), nch, s));
                RB_CU(launch_forward_reduce(G, F.f[w], W.at<float2>(W.L.fwd), nch, dw, wts + (size_t)w * ne2,
                                            part + (size_t)w * 256, s));
            }
        }
        RB_CU(launch_sum_partials(part, n_freq * 256, dbl, DBL_CG_PAP + k, 1.0, 0, s));
        // q = sum_w Re B_w^H W B_w p
        if (tc) {
            RB_CU(launch_adjoint_tc(G, W.at<void>(W.L.aimg), F, W.at<void>(W.L.tcimg), W.at<float2>(W.L.gscr),
                                    tc_ctas(), nullptr, nullptr, q, nullptr, cnt, s, (params->tune >> 2) & 3));
        } else {
            RB_CU(launch_adjoint_simt(G, tables, c_inout, F, d, wts, nullptr, nullptr, q, nullptr, cnt, s));
        }
        RB_CU(launch_cg_step(G, hsum, precond, k, x, r, p, q, vpart, dbl, s));
    }
    if (cg_hist_out) RB_CU(launch_cg_history(dbl, cg_iters, cg_hist_out, s));
    RB_CU(mark(RB_STAGE_FORWARD, 1));
    RB_CU(mark(RB_STAGE_APPLY, 0));
    RB_CU(launch_update(G, c_inout, gsum, hsum, x, dc_out, vpart, dbl, cnt, diag_out, params->eps_rel, RB_STEP_DIAG,
                        1, s, limit_word));
    RB_CU(mark(RB_STAGE_APPLY, 1));
    return RB_OK;
}

rb_status rb_tof_times(const rb_geometry* geom, const float* c, const float* alpha0, double* t_out,
                       uint8_t* linked_out, void* ws, size_t ws_bytes, rb_stream stream) {
    if (!geom || !c || !alpha0 || !t_out) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    Ws W;
    rb_status st = check_ws(geom, 1, RB_PREC_FP32, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    rb_ray_end* ends = W.at<rb_ray_end>(W.L.ends);
    RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
    RB_CU(launch_elem_positions(G, exy, s));
    RB_CU(launch_fields(G, c, alpha0, W.at<float4>(W.L.cells), s));
    RB_CU(launch_trace(G, W.at<float4>(W.L.cells), ends, nullptr, nullptr, nullptr, nullptr, nullptr, cnt, s));
    RB_CU(launch_tof_link(G, c, ends, W.at<void>(W.L.tof), linked_out, s));
    RB_CU(launch_tof_times_out(G, W.at<void>(W.L.tof), t_out, s));
    return RB_OK;
}

rb_status rb_tof_invert(const rb_geometry* geom, float* c_inout, const float* alpha0, const double* t_obs,
                        const uint8_t* obs_linked, int32_t n_iter, double* resid_out, void* ws, size_t ws_bytes,
                        rb_stream stream) {
    if (!geom || !c_inout || !alpha0 || !t_obs || !obs_linked) return RB_ERR_ARG;
    if (n_iter < 1 || n_iter > RB_MAX_TOF_ITERS) return RB_ERR_ARG;
    if (!geom_ok(geom)) return RB_ERR_SHAPE;
    Ws W;
    rb_status st = check_ws(geom, 1, RB_PREC_FP32, ws, ws_bytes, &W);
    if (st != RB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* exy = W.at<float4>(W.L.elem_xy);
    uint32_t* cnt = W.at<uint32_t>(W.L.counters);
    const GeoDev G = make_geo(geom, exy);
    rb_ray_end* ends = W.at<rb_ray_end>(W.L.ends);
    float4* cells = W.at<float4>(W.L.cells);
    void* tw = W.at<void>(W.L.tof);
    Vtx* verts = W.at<Vtx>(W.L.verts);
    double* part = W.at<double>(W.L.part);
    RB_CU(cudaMemsetAsync(cnt, 0, CNT_N * 4, s));
    RB_CU(launch_elem_positions(G, exy, s));
    for (int k = 0; k <= n_iter; ++k) {
        const bool last = k == n_iter;
        RB_CU(launch_fields(G, c_inout, alpha0, cells, s));
        RB_CU(launch_trace(G, cells, ends, nullptr, nullptr, nullptr, last ? nullptr : (void*)verts, nullptr, cnt, s));
        RB_CU(launch_tof_link(G, c_inout, ends, tw, nullptr, s));
        if (resid_out) RB_CU(launch_tof_resid(G, tw, t_obs, obs_linked, part, resid_out + k, s));
        if (!last) RB_CU(launch_tof_step(G, verts, ends, tw, t_obs, obs_linked, c_inout, s));
    }
    return RB_OK;
}

}  // extern "C"
