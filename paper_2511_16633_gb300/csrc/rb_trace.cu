// Ray fans and first-arrival gridding, fused in one kernel.
//
// Physics (Sec. 2): the Eikonal equation (Eq. 6) is integrated along its
// characteristics and the Transport equation (Eq. 7) through the dynamic
// ray-tracing pair (Q, P); in arclength s
//   x' = cos th, y' = sin th, th' = (c_x sin th - c_y cos th) / c,
//   T' = 1/c, Q' = c P, P' = -(c_nn / c^2) Q, L' = alpha0,
// c_nn = c_xx sin^2 th - 2 c_xy sin th cos th + c_yy cos^2 th, by classical RK4
// with fixed step ds from the element position, take-off angle
// th0 = phi_t + pi/2 + (i + 1/2) pi / n_rays, T = Q = L = 0, P = 1/c(x_t).  A ray
// ends at the first step k >= 1 with |x_k| >= R; its last vertex is the
// segment's crossing of the ring with every state component interpolated
// linearly.  KMAH index: sign changes of Q from the second step on.
//
// Gridding ("back-propagation of ray parameters", Sec. 5): neighbouring rays
// i, i+1 and steps k-1, k bound a quad split into triangles
// {(i,k-1),(i+1,k-1),(i+1,k)} and {(i,k-1),(i+1,k),(i,k)}; a ray that has
// ended repeats its last vertex.  Support pixels inside a triangle get the
// barycentric interpolation of T_res = T - |x - x_t|/c_ref, Q, L and the
// KMAH index of the heaviest vertex; the smallest T_res wins (ties: smallest
// triangle id).
//
// GB300 mapping: three kernels.  k_trace runs one thread per ray (field samples
// from the 128-byte cell records of rb_fields.cu, kept in registers while a ray
// stays in its cell) and streams every vertex out (32 B).  k_raster gives each
// thread a tube and a block of 8 steps, so the rasterisation runs at full
// occupancy; every covered pixel gets a fire-and-forget 64-bit atomic min of
// (T_res key, triangle id) in an 8-byte key array.  k_resolve then reads the
// winning triangle id of every hit pixel, fetches that triangle's vertices and
// writes the table record (Q, L and the KMAH index) and/or the synthesis record,
// and counts the support pixels no triangle covered.
// Positions, the direction and the traveltime T are float pairs (compensated
// sums; the vertex residual T - |x - x_t|/c_ref is formed in float pairs too),
// which keeps the Green's-function phase w T accurate at MHz frequencies without
// the (slow) FP64 pipe.
#include "rb_internal.cuh"

namespace {

struct Cache {
    float fi, fj;   // cell indices of the cached record (as floats; -1 = none)
    float4 r[7];    // field pairs (c, c_x), (c_y, c_xx), (c_xy, c_yy) as {a, a', b, b'}, {c, c', d, d'}; alpha0
};

struct Deriv { float x, y, th, t, q, p, l; };

// Bilinear samples of c, c_x, c_y, c_xx, c_xy, c_yy, alpha0 at (px, py).  The cell
// record holds per field the coefficients (a, b, c, d) of a + b u + c v + d u v over the
// cell's unit square, paired fields side by side (rb_fields.cu), so each pair takes three
// packed two-lane FMAs (same operations and rounding as three scalar ones per field).
// The cell indices stay floats (floorf), and the record is reloaded only when the ray
// changes cell.
__device__ __forceinline__ void sample(const GeoDev& G, const float4* __restrict__ cells, Cache& cc, float px, float py,
                                       float f[7]) {
    const float u = fminf(fmaxf(fmaf(px, G.inv_h, G.cxg), 0.f), G.fxmax);
    const float v = fminf(fmaxf(fmaf(py, G.inv_h, G.cyg), 0.f), G.fymax);
    const float fi = fminf(floorf(u), G.fxmax - 1.f), fj = fminf(floorf(v), G.fymax - 1.f);
    const float fu = u - fi, fv = v - fj;
    if (fi != cc.fi || fj != cc.fj) {
        const float4* p = cells + ((size_t)(int)fj * (size_t)(G.nx - 1) + (size_t)(int)fi) * 8;
#pragma unroll
        for (int k = 0; k < 7; ++k) cc.r[k] = __ldg(p + k);
        cc.fi = fi;
        cc.fj = fj;
    }
    const float uv = fu * fv;
    const float2 u2 = make_float2(fu, fu), v2 = make_float2(fv, fv), w2 = make_float2(uv, uv);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 ab = cc.r[2 * k], cd = cc.r[2 * k + 1];
        const float2 s = __ffma2_rn(make_float2(cd.z, cd.w), w2,
                                    __ffma2_rn(make_float2(cd.x, cd.y), v2,
                                               __ffma2_rn(make_float2(ab.z, ab.w), u2, make_float2(ab.x, ab.y))));
        f[2 * k] = s.x;
        f[2 * k + 1] = s.y;
    }
    const float4 q = cc.r[6];
    f[6] = fmaf(q.w, uv, fmaf(q.z, fv, fmaf(q.y, fu, q.x)));
}

// sin and cos of a ray angle (|x| < 1e4 rad), inline and branch-light: Cody-Waite
// reduction by pi/2 in three float parts (r = x - k pi/2 to ~1e-9 absolute for these
// arguments), Taylor polynomials on |r| <= pi/4 (sin to r^11, cos to r^12: truncation
// below 1e-9), then the quadrant.  Used for the anchor angle instead of the library
// call, whose large-argument path, inlined into the step loop, cost registers and
// issue slots on every step.
__device__ __forceinline__ void ray_sincos(float x, float* s, float* c) {
    const float k = rintf(x * 0.636619772367581343f);   // x / (pi / 2)
    float r = fmaf(-k, 1.5707962513e+00f, x);             // pi/2 = p1 + p2 + p3
    r = fmaf(-k, 7.5497894159e-08f, r);
    r = fmaf(-k, 5.3903029534e-15f, r);
    const float r2 = r * r;
    // sin r = r (1 - r^2/3! + r^4/5! - ...), cos r = 1 - r^2/2! + r^4/4! - ...
    float ps = fmaf(r2, -2.50521083854e-08f, 2.75573192240e-06f);   // -1/11!, 1/9!
    ps = fmaf(r2, ps, -1.98412698413e-04f);                           // -1/7!
    ps = fmaf(r2, ps, 8.33333333333e-03f);                            // 1/5!
    ps = fmaf(r2, ps, -1.66666666667e-01f);                           // -1/3!
    const float sn = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, 2.08767569879e-09f, -2.75573192240e-07f);     // 1/12!, -1/10!
    pc = fmaf(r2, pc, 2.48015873016e-05f);                            // 1/8!
    pc = fmaf(r2, pc, -1.38888888889e-03f);                           // -1/6!
    pc = fmaf(r2, pc, 4.16666666667e-02f);                            // 1/4!
    pc = fmaf(r2, pc, -0.5f);                                         // -1/2!
    const float cs = fmaf(r2, pc, 1.0f);
    const int q = (int)k & 3;
    const float ss = (q & 1) ? cs : sn, cc = (q & 1) ? sn : cs;
    *s = (q & 2) ? -ss : ss;
    *c = ((q + 1) & 2) ? -cc : cc;
}

// cos/sin of (th_hi + d) from cos/sin of th_hi and a small d (Taylor to d^7).
__device__ __forceinline__ void rotate(float C0, float S0, float th_hi, float d, float& c, float& s) {
    if (fabsf(d) < 0.2f) {
        const float d2 = d * d;
        const float cd = 1.f - 0.5f * d2 * (1.f - d2 * (1.f / 12.f) * (1.f - d2 * (1.f / 30.f)));
        const float sd = d * (1.f - d2 * (1.f / 6.f) * (1.f - d2 * (1.f / 20.f) * (1.f - d2 * (1.f / 42.f))));
        c = C0 * cd - S0 * sd;
        s = S0 * cd + C0 * sd;
    } else {
        // a turn of 0.2 rad within half a step (gradients far beyond tissue): the hardware
        // approximation (~1e-6 absolute), small enough not to weigh on the common path
        __sincosf(th_hi + d, &s, &c);
    }
}

__device__ __forceinline__ Deriv eval_stage(const GeoDev& G, const float4* __restrict__ cells, Cache& cc,
                                            float xh, float xl, float yh, float yl, float Ca, float Sa, float tha,
                                            float dth, float q, float p,
                                            float a, const Deriv& kp) {
    const float ox = fmaf(a, kp.x, xl), oy = fmaf(a, kp.y, yl);
    const float px = xh + ox, py = yh + oy;
    float cth, sth;
    rotate(Ca, Sa, tha, fmaf(a, kp.th, dth), cth, sth);
    const float qs = fmaf(a, kp.q, q), ps = fmaf(a, kp.p, p);
    float f[7];
    sample(G, cells, cc, px, py, f);
    const float c = f[0];
    const float rc = __fdividef(1.0f, c);   // ~2 ulp: far below the RK4 truncation error
    Deriv d;
    d.x = cth;
    d.y = sth;
    d.th = (f[1] * sth - f[2] * cth) * rc;
    d.t = rc;   // T' = 1 / c (the residual T - |x - x_t| / c_ref is formed per vertex)
    d.q = c * ps;
    const float cnn = f[3] * sth * sth - 2.f * f[4] * sth * cth + f[5] * cth * cth;
    d.p = -(cnn * rc * rc) * qs;
    d.l = f[6];
    return d;
}

__device__ __forceinline__ void comp_add(float& hi, float& lo, float inc) {
    DF s = df_two_sum(hi, inc);
    DF r = df_fast_two_sum(s.hi, __fadd_rn(lo, s.lo));
    hi = r.hi;
    lo = r.lo;
}

// Exact ring test of a float-pair position, in double.  Not inlined: GB300's FP64
// pipe is slow, and an inlined copy would be predicated into every RK4 step
// instead of running only on the few steps the float screen lets through.
__device__ __noinline__ bool outside_ring(float xh, float xl, float yh, float yl, double R) {
    const double dx = (double)xh + (double)xl, dy = (double)yh + (double)yl;
    return dx * dx + dy * dy >= R * R;
}

__device__ __forceinline__ double exit_lambda(double ax, double ay, double bx, double by, double R) {
    const double dx = bx - ax, dy = by - ay;
    const double qa = dx * dx + dy * dy;
    const double qb = 2.0 * (ax * dx + ay * dy);
    const double qc = ax * ax + ay * ay - R * R;
    double disc = qb * qb - 4.0 * qa * qc;
    if (disc < 0.0) disc = 0.0;
    const double sq = sqrt(disc);
    double lam;
    if (qb >= 0.0) {
        const double den = qb + sq;
        lam = den > 0.0 ? -2.0 * qc / den : 0.0;
    } else {
        lam = (-qb + sq) / (2.0 * qa);
    }
    return fmin(fmax(lam, 0.0), 1.0);
}

// Geometry of one ray-tube quad relative to its vertex A0 (float-pair differences):
// triangle T0 = (A0, B0, B1) spans edge vectors b0, b1; T1 = (A0, B1, A1) spans b1, a1.
// Twice the signed areas are exactly zero when two vertices coincide (frozen rays).
struct Quad {
    float b0x, b0y, b1x, b1y, a1x, a1y;
    float i0, i1;   // reciprocal doubled areas (0 for a degenerate triangle)
    bool t0, t1;
};

__device__ __forceinline__ float rel(float vh, float vl, float oh, float ol) {
    return __fadd_rn(__fsub_rn(vh, oh), __fsub_rn(vl, ol));
}

// Barycentric weights of the point A0 + (dx, dy) in the triangle with edge vectors
// (ux, uy), (vx, vy) from A0 and reciprocal doubled area inv: w = (wa, wb, wc) for
// (A0, A0 + u, A0 + v).
__device__ __forceinline__ void bary(float ux, float uy, float vx, float vy, float inv, float dx, float dy, float& wa,
                                     float& wb, float& wc) {
    wb = __fmul_rn(__fsub_rn(__fmul_rn(dx, vy), __fmul_rn(dy, vx)), inv);
    wc = __fmul_rn(__fsub_rn(__fmul_rn(ux, dy), __fmul_rn(uy, dx)), inv);
    wa = __fsub_rn(__fsub_rn(1.f, wb), wc);
}

__device__ __forceinline__ float interp(float wa, float wb, float wc, float a, float b, float c) {
    return __fadd_rn(__fadd_rn(__fmul_rn(wa, a), __fmul_rn(wb, b)), __fmul_rn(wc, c));
}

// Keep the smaller 64-bit key (T_res key << 32 | triangle id << 8) of a pixel: the
// order of the first 8 bytes of a table record ({tag, tkey} little-endian).  No
// value is returned, so the warp never waits.
__device__ __forceinline__ void key_min(unsigned long long* dst, uint64_t key) {
    asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(dst), "l"(key) : "memory");
}

// Rasterise one ray-tube quad: triangles T0 (id base) and T1 (id base + 1).  One
// pixel box (pixel centres inside the quad's bounding box, cut to the support
// disc row by row) serves both triangles; where both contain a pixel the smaller
// T_res (then T0) is offered.  Along a row the weights and T_res are affine in
// the pixel index: they are evaluated at the row's first pixel and then stepped
// by their exact per-pixel increments (a few ulps of drift over a box).
__device__ __forceinline__ void raster_quad(const GeoDev& G, const Vtx& A0, const Vtx& A1, const Vtx& B0, const Vtx& B1,
                                            uint32_t base, uint32_t fl, unsigned long long* __restrict__ tab,
                                            const short2* __restrict__ supp) {
    // edge vectors first: most quads are about one pixel, and a box with no pixel centre
    // ends here before the areas and their reciprocals are formed
    Quad Q;
    Q.b0x = rel(B0.xh, B0.xl, A0.xh, A0.xl);
    Q.b0y = rel(B0.yh, B0.yl, A0.yh, A0.yl);
    Q.b1x = rel(B1.xh, B1.xl, A0.xh, A0.xl);
    Q.b1y = rel(B1.yh, B1.yl, A0.yh, A0.yl);
    Q.a1x = rel(A1.xh, A1.xl, A0.xh, A0.xl);
    Q.a1y = rel(A1.yh, A1.yl, A0.yh, A0.yl);
    // tight box of pixel centres (index space), with a 1e-3 px guard
    const float ua = fmaf(A0.xh, G.inv_h, G.cxg) + A0.xl * G.inv_h;
    const float va = fmaf(A0.yh, G.inv_h, G.cyg) + A0.yl * G.inv_h;
    const float xmin = fminf(fminf(0.f, Q.b0x), fminf(Q.b1x, Q.a1x)), xmax = fmaxf(fmaxf(0.f, Q.b0x), fmaxf(Q.b1x, Q.a1x));
    const float ymin = fminf(fminf(0.f, Q.b0y), fminf(Q.b1y, Q.a1y)), ymax = fmaxf(fmaxf(0.f, Q.b0y), fmaxf(Q.b1y, Q.a1y));
    // a non-finite vertex (only from a non-physical sound speed, e.g. zero or infinite) would
    // give a box over the whole grid: such a quad covers nothing
    if (!isfinite(ua + va + xmin + xmax + ymin + ymax)) return;
    const int bx0 = max(0, (int)ceilf(fmaf(xmin, G.inv_h, ua) - 1e-3f));
    const int bx1 = min(G.nx - 1, (int)floorf(fmaf(xmax, G.inv_h, ua) + 1e-3f));
    const int iy0 = max(0, (int)ceilf(fmaf(ymin, G.inv_h, va) - 1e-3f));
    const int iy1 = min(G.ny - 1, (int)floorf(fmaf(ymax, G.inv_h, va) + 1e-3f));
    if (bx0 > bx1 || iy0 > iy1) return;
    {
        // doubled areas of T0 and T1, with the hardware reciprocal: these weights only decide coverage and
        // the residual offered as the key; the table record's weights are formed exactly
        // by the resolve pass
        const float ar0 = __fsub_rn(__fmul_rn(Q.b0x, Q.b1y), __fmul_rn(Q.b0y, Q.b1x));
        const float ar1 = __fsub_rn(__fmul_rn(Q.b1x, Q.a1y), __fmul_rn(Q.b1y, Q.a1x));
        Q.t0 = ar0 != 0.f;
        Q.t1 = ar1 != 0.f;
        Q.i0 = Q.t0 ? __fdividef(1.0f, ar0) : 0.f;
        Q.i1 = Q.t1 ? __fdividef(1.0f, ar1) : 0.f;
    }
    if (!Q.t0 && !Q.t1) return;
    const float tol = -1e-6f;
    // per-pixel (x) increments of the weights of T0 = (A0; u = b0, v = b1) and T1 = (A0; u = b1, v = a1)
    const float h = G.h;
    const float db0 = Q.b1y * Q.i0 * h, dc0 = -Q.b0y * Q.i0 * h;
    const float db1 = Q.a1y * Q.i1 * h, dc1 = -Q.b1y * Q.i1 * h;
    const float tb0 = B0.t - A0.t, tc0 = B1.t - A0.t;    // T = A0.t + wb (Tb - Ta) + wc (Tc - Ta)
    const float tb1 = B1.t - A0.t, tc1 = A1.t - A0.t;
    const DF X0 = df_pixel_coord(bx0, G.cxg, G.h_hi, G.h_lo);
    const float dx0 = rel(X0.hi, X0.lo, A0.xh, A0.xl);
    for (int iy = iy0; iy <= iy1; ++iy) {
        const short2 sr = supp[iy];   // support disc columns of this row
        const int ix0 = max(bx0, (int)sr.x), ix1 = min(bx1, (int)sr.y);
        if (ix0 > ix1) continue;
        const DF Y = df_pixel_coord(iy, G.cyg, G.h_hi, G.h_lo);
        const float dy = rel(Y.hi, Y.lo, A0.yh, A0.yl);
        const float dx = dx0 + (float)(ix0 - bx0) * h;
        float wb0 = 0.f, wc0 = 0.f, wb1 = 0.f, wc1 = 0.f, wa;
        if (Q.t0) bary(Q.b0x, Q.b0y, Q.b1x, Q.b1y, Q.i0, dx, dy, wa, wb0, wc0);
        if (Q.t1) bary(Q.b1x, Q.b1y, Q.a1x, Q.a1y, Q.i1, dx, dy, wa, wb1, wc1);
        size_t o = (size_t)iy * G.nx + ix0;
        for (int ix = ix0; ix <= ix1; ++ix, ++o) {
            const bool in0 = Q.t0 && wb0 >= tol && wc0 >= tol && (1.f - wb0 - wc0) >= tol;
            const bool in1 = Q.t1 && wb1 >= tol && wc1 >= tol && (1.f - wb1 - wc1) >= tol;
            if (in0 || in1) {
                const float tr0 = fmaf(wb0, tb0, fmaf(wc0, tc0, A0.t));
                const float tr1 = fmaf(wb1, tb1, fmaf(wc1, tc1, A0.t));
                const bool use1 = in1 && (!in0 || tr1 < tr0);
                const uint32_t id = use1 ? base + 1u : base;
                key_min(tab + o, ((uint64_t)f2key(use1 ? tr1 : tr0) << 32) | ((uint64_t)id << 8) | fl);
            }
            wb0 += db0;
            wc0 += dc0;
            wb1 += db1;
            wc1 += dc1;
        }
    }
}

// q / d and q % d for q < 2^31, d >= 1, with m = floor(2^32 / d): the high word of q m
// is the quotient or one less.
__device__ __forceinline__ void udivmod(uint32_t q, uint32_t d, uint32_t m, uint32_t& quo, uint32_t& rem) {
    uint32_t x = __umulhi(q, m);
    uint32_t r = q - x * d;
    if (r >= d) {
        ++x;
        r -= d;
    }
    quo = x;
    rem = r;
}

__device__ __forceinline__ size_t vidx(const GeoDev& G, int t, int k, int i) { return vtx_index(G, t, k, i); }

__device__ __forceinline__ void put_vtx(Vtx* dst, const Vtx& v) {
    float4* d = reinterpret_cast<float4*>(dst);
    d[0] = make_float4(v.xh, v.xl, v.yh, v.yl);
    d[1] = make_float4(v.t, v.q, v.l, __int_as_float(v.k));
}

// One thread per ray: RK4 from the element to the ring, the end record, and (when
// verts is set) every vertex into the vertex stream for the rasteriser.
constexpr int TRACE_GR = 8;   // rays of one fan side by side in a warp (measured: 1, 2, 4, 8, 16)
__global__ void __launch_bounds__(128) k_trace(GeoDev G, const float4* __restrict__ cells, rb_ray_end* __restrict__ ends,
                                               rb_rays S, int write_samples, Vtx* __restrict__ verts,
                                               uint32_t* __restrict__ counters, uint32_t* __restrict__ fan_len) {
    // a warp takes TRACE_GR neighbouring rays of 32 / TRACE_GR fans: rays of alike take-off
    // angles (so alike lengths: the lanes finish together) that share field cells
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long qg = u / ((long long)TRACE_GR * G.n_elem), rg = u % ((long long)TRACE_GR * G.n_elem);
    const int t = (int)(rg / TRACE_GR), i = (int)(qg * TRACE_GR + rg % TRACE_GR);
    if (i >= G.n_rays) return;
    const bool valid = true, owner = true;
    const bool put = verts != nullptr;

    DF xs, ys;
    elem_pos(G, t, xs, ys);
    const double xs_d = (double)xs.hi + (double)xs.lo, ys_d = (double)ys.hi + (double)ys.lo;
    const double th0 = 2.0 * RB_PI_D * (double)t / (double)G.n_elem + 0.5 * RB_PI_D +
                       ((double)i + 0.5) * RB_PI_D / (double)G.n_rays;
    const DF thd = df_from_double(th0);

    Cache cc;
    cc.fi = -1.f;
    cc.fj = -1.f;
    float f0[7];
    sample(G, cells, cc, xs.hi + xs.lo, ys.hi + ys.lo, f0);

    float xh = xs.hi, xl = xs.lo, yh = ys.hi, yl = ys.lo, thh = thd.hi, thl = thd.lo;
    float tha = thh, Ca, Sa;
    sincosf(tha, &Sa, &Ca);
    float trh = 0.f, trl = 0.f;   // T as a float pair (compensated sum of the RK4 increments)
    float q = 0.f, p = 1.0f / f0[0], l = 0.f;
    int kap = 0;
    bool alive = valid;

    Vtx cur{xh, xl, yh, yl, 0.f, 0.f, 0.f, 0};
    const size_t sbase = ((size_t)t * G.n_rays + (valid ? i : 0)) * (size_t)(G.max_steps + 1);
    if (write_samples && valid) {
        S.vx[sbase] = xh + xl;
        S.vy[sbase] = yh + yl;
        S.vt[sbase] = 0.0;
        S.vq[sbase] = 0.f;
        S.vl[sbase] = 0.f;
        S.vkappa[sbase] = 0;
    }
    if (put) put_vtx(verts + vidx(G, t, 0, i), cur);
    const float ds = G.ds, a2 = 0.5f * G.ds, ds6 = G.ds * (1.0f / 6.0f);

    for (int k = 1; k <= G.max_steps; ++k) {
        if (!alive) break;
        if (alive) {
            // direction relative to the anchor angle tha (cos / sin exact there); the
            // anchor follows the ray whenever it has turned by more than 0.05 rad
            // a loop rather than an if: the compiler keeps it a branch instead of evaluating
            // the refresh on every step (it runs at most once)
            while (fabsf(thh - tha) > 0.05f) {
                tha = thh;
                ray_sincos(tha, &Sa, &Ca);
            }
            const float dth = (thh - tha) + thl;
            const Deriv z{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const Deriv k1 = eval_stage(G, cells, cc, xh, xl, yh, yl, Ca, Sa, tha, dth, q, p, 0.f, z);
            const Deriv k2 = eval_stage(G, cells, cc, xh, xl, yh, yl, Ca, Sa, tha, dth, q, p, a2, k1);
            const Deriv k3 = eval_stage(G, cells, cc, xh, xl, yh, yl, Ca, Sa, tha, dth, q, p, a2, k2);
            const Deriv k4 = eval_stage(G, cells, cc, xh, xl, yh, yl, Ca, Sa, tha, dth, q, p, ds, k3);
            const float ix = ds6 * (k1.x + 2.f * k2.x + 2.f * k3.x + k4.x);
            const float iy = ds6 * (k1.y + 2.f * k2.y + 2.f * k3.y + k4.y);
            const float ith = ds6 * (k1.th + 2.f * k2.th + 2.f * k3.th + k4.th);
            const float it = ds6 * (k1.t + 2.f * k2.t + 2.f * k3.t + k4.t);
            const float iq = ds6 * (k1.q + 2.f * k2.q + 2.f * k3.q + k4.q);
            const float ip = ds6 * (k1.p + 2.f * k2.p + 2.f * k3.p + k4.p);
            const float il = ds6 * (k1.l + 2.f * k2.l + 2.f * k3.l + k4.l);
            float nxh = xh, nxl = xl, nyh = yh, nyl = yl, nthh = thh, nthl = thl;
            comp_add(nxh, nxl, ix);
            comp_add(nyh, nyl, iy);
            comp_add(nthh, nthl, ith);
            const float nq = q + iq, np = p + ip, nl = l + il;
            // exit test: float screen, then double decision
            const float fx = nxh + nxl, fy = nyh + nyl;
            bool out = false;
            if (fx * fx + fy * fy >= G.R2 * (1.0f - 4e-6f)) out = outside_ring(nxh, nxl, nyh, nyl, G.R_d);
            if (out) {
                const double ax = (double)xh + (double)xl, ay = (double)yh + (double)yl;
                const double bx = (double)nxh + (double)nxl, by = (double)nyh + (double)nyl;
                const double lam = exit_lambda(ax, ay, bx, by, G.R_d);
                const float lf = (float)lam;
                const double ex = ax + lam * (bx - ax), ey = ay + lam * (by - ay);
                const double tt = (double)trh + (double)trl;
                const double et = tt + lam * (double)it;
                const double eth = ((double)thh + (double)thl) + lam * (((double)nthh + (double)nthl) - ((double)thh + (double)thl));
                const float eq = q + lf * (nq - q), ep = p + lf * (np - p), el = l + lf * (nl - l);
                const int ek = kap + ((k >= 2 && signbit(eq) != signbit(q)) ? 1 : 0);
                const DF exd = df_from_double(ex), eyd = df_from_double(ey);
                xh = exd.hi; xl = exd.lo; yh = eyd.hi; yl = eyd.lo;
                const DF etd = df_from_double(et);
                q = eq; p = ep; l = el; kap = ek; trh = etd.hi; trl = etd.lo;
                alive = false;
                if (owner) {
                    const double ddx = ex - xs_d, ddy = ey - ys_d;
                    rb_ray_end e;
                    e.t = et;
                    e.t_res = et - sqrt(ddx * ddx + ddy * ddy) * (1.0 / G.c_ref_d);
                    e.x = ex;
                    e.y = ey;
                    e.theta = (float)eth;
                    e.q = eq;
                    e.p = ep;
                    e.l = el;
                    e.kappa = ek;
                    e.n_vert = k + 1;
                    ends[(size_t)t * G.n_rays + i] = e;
                    if (fan_len) atomicMax(fan_len + t, (uint32_t)(k + 1));
                }
            } else {
                if (k >= 2 && signbit(nq) != signbit(q)) ++kap;
                xh = nxh; xl = nxl; yh = nyh; yl = nyl; thh = nthh; thl = nthl;
                comp_add(trh, trl, it);
                q = nq; p = np; l = nl;
                if (k == G.max_steps) {
                    alive = false;
                    if (owner) {
                        const double ex = (double)xh + (double)xl, ey = (double)yh + (double)yl;
                        const double ddx = ex - xs_d, ddy = ey - ys_d;
                        rb_ray_end e;
                        const double tt = (double)trh + (double)trl;
                        e.t = tt;
                        e.t_res = tt - sqrt(ddx * ddx + ddy * ddy) * (1.0 / G.c_ref_d);
                        e.x = ex;
                        e.y = ey;
                        e.theta = thh + thl;
                        e.q = q;
                        e.p = p;
                        e.l = l;
                        e.kappa = kap;
                        e.n_vert = -1;
                        ends[(size_t)t * G.n_rays + i] = e;
                        atomicAdd(counters + CNT_LOST, 1u);
                        if (fan_len) atomicMax(fan_len + t, (uint32_t)(G.max_steps + 1));
                    }
                }
            }
            if (put) {
                // vertex residual T - |x - x_t| / c_ref in float pairs
                const DF dx = df_sub(DF{xh, xl}, xs), dy = df_sub(DF{yh, yl}, ys);
                const DF d2 = df_add(df_sqr(dx), df_sqr(dy));
                const DF dist = d2.hi > 0.f ? df_sqrt(d2) : DF{0.f, 0.f};
                const DF tr = df_sub(DF{trh, trl}, df_mul(dist, DF{G.inv_cref, G.inv_cref_lo}));
                cur = Vtx{xh, xl, yh, yl, tr.hi + tr.lo, q, l, kap};
                put_vtx(verts + vidx(G, t, k, i), cur);
            }
            if (write_samples) {
                const size_t o = sbase + (size_t)k;
                const double vx = (double)xh + (double)xl, vy = (double)yh + (double)yl;
                S.vx[o] = (float)vx;
                S.vy[o] = (float)vy;
                S.vt[o] = (double)trh + (double)trl;
                S.vq[o] = q;
                S.vl[o] = l;
                S.vkappa[o] = kap;
            }
        }
    }
}

// Index of the last vertex of ray i of fan t: the exit vertex, or max_steps for a
// lost ray.  Past it the ray repeats that vertex, as in the rasteriser.
__device__ __forceinline__ int last_vertex(const GeoDev& G, const rb_ray_end* __restrict__ ends, int t, int i) {
    const int nv = ends[(size_t)t * G.n_rays + i].n_vert;
    return nv > 0 ? nv - 1 : G.max_steps;
}

__device__ __forceinline__ Vtx get_vtx(const Vtx* __restrict__ src) {
    const float4* s = reinterpret_cast<const float4*>(src);
    const float4 a = __ldg(s), b = __ldg(s + 1);
    return Vtx{a.x, a.y, a.z, a.w, b.x, b.y, b.z, __float_as_int(b.w)};
}

// Rasteriser: warp (t, i, kc) rasterises the quads k = 32 kc + 1 .. 32 kc + 32 of tube
// (i, i + 1) of fan t from the vertex stream, one per lane, up to the later of the two
// rays' last vertices (beyond it both triangles are degenerate).  Neighbouring quads
// along a tube are alike in size, so the lanes' pixel loops are of similar length (32
// tubes at the same step, the other way round, differ far more where the medium bends
// the rays); each lane's four vertices are 32-byte loads, shared with the next lane
// through L1.
constexpr int KW = 32;
constexpr int KB = 8;   // quads per thread of the tube-major mapping
#ifndef RASTER_ALONG_K_MIN_PX
#define RASTER_ALONG_K_MIN_PX 4.0   // tube width (pixels, across the ring) from which warps run along the tubes
#endif

// Low bits of a quad's key: bit 0 when ray i has ended before step k (its vertices
// there repeat its last one), bit 1 the same for ray i + 1.  The resolve pass reads
// the rays' ends only for such quads.
__device__ __forceinline__ uint32_t clamp_flags(int k, int la, int lb) {
    return (uint32_t)(k > la) | ((uint32_t)(k > lb) << 1);
}

// The last quad index any tube of fan t reaches: its longest ray's last vertex (the
// tracer's per-fan maximum of the vertex counts), at most max_steps.
__device__ __forceinline__ int fan_last_quad(const GeoDev& G, const uint32_t* __restrict__ fan_len, int t) {
    const uint32_t nv = __ldg(fan_len + t);
    return nv == 0u ? 0 : (int)min(nv - 1u, (uint32_t)G.max_steps);
}

// Columns [lo, hi] of row iy inside the support disc (2 ix - (nx - 1))^2 +
// (2 iy - (ny - 1))^2 <= r2max, exact in integers; lo > hi for an empty row.
__device__ __forceinline__ short2 support_row(const GeoDev& G, int iy) {
    const int jy = 2 * iy - (G.ny - 1);
    const long long rem = G.r2max - (long long)jy * jy;
    if (rem < 0) return make_short2(1, 0);
    int sj = (int)sqrtf((float)rem);
    while ((long long)(sj + 1) * (sj + 1) <= rem) ++sj;
    while (sj > 0 && (long long)sj * sj > rem) --sj;
    const int lo = max(0, (G.nx - 1 - sj + 1) >> 1), hi = min(G.nx - 1, (G.nx - 1 + sj) >> 1);
    return make_short2((short)lo, (short)hi);
}

// ALONG_K: a warp takes 32 consecutive quads of one tube (one per lane) -- for fans whose
// tubes span several pixels, where neighbouring quads of a tube are alike in size.
// Otherwise a thread takes 8 consecutive quads of one tube and a warp 32 neighbouring
// tubes at the same steps -- for fans finer than the grid, whose quads mostly cover at
// most one pixel, where the vertex loads (contiguous across tubes) set the pace.
// Threads per CTA: 128 along the tubes (smaller blocks leave room sooner for the update's
// linking kernels beside the rasteriser), 256 across them.
template <bool ALONG_K>
constexpr int raster_threads() { return ALONG_K ? 128 : 256; }

template <bool ALONG_K>
__global__ void __launch_bounds__(raster_threads<ALONG_K>()) k_raster(GeoDev G, const Vtx* __restrict__ verts,
                                                const rb_ray_end* __restrict__ ends, unsigned long long* __restrict__ keys,
                                                const uint32_t* __restrict__ fan_len, uint32_t nt_magic) {
    extern __shared__ short2 s_supp[];   // [ny]
    for (int iy = threadIdx.x; iy < G.ny; iy += blockDim.x) s_supp[iy] = support_row(G, iy);
    __syncthreads();
    const int NT = G.n_rays - 1;
    const uint32_t KQ = (uint32_t)(G.max_steps + 1);
    if (ALONG_K) {
        const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
        // fans t = blockIdx.y + j gridDim.y; within a fan, warp item = kc NT + i, up to the
        // fan's longest ray (quads k <= its last vertex)
        for (int t = blockIdx.y; t < G.n_elem; t += gridDim.y) {
        const int kmax = fan_last_quad(G, fan_len, t);
        const int per_fan = ((kmax + KW - 1) / KW) * NT;   // < 2^31 (the triangle ids fit 24 bits)
        for (int item = blockIdx.x * wpb + wib; item < per_fan; item += gridDim.x * wpb) {
            uint32_t ukc, ui;
            udivmod((uint32_t)item, (uint32_t)NT, nt_magic, ukc, ui);
            const int i = (int)ui;
            const int la = last_vertex(G, ends, t, i), lb = last_vertex(G, ends, t, i + 1);
            const int k = (int)ukc * KW + lane + 1;
            if (k > max(la, lb)) continue;
            const Vtx A0 = get_vtx(verts + vidx(G, t, min(k - 1, la), i));
            const Vtx B0 = get_vtx(verts + vidx(G, t, min(k - 1, lb), i + 1));
            const Vtx A1 = get_vtx(verts + vidx(G, t, min(k, la), i));
            const Vtx B1 = get_vtx(verts + vidx(G, t, min(k, lb), i + 1));
            raster_quad(G, A0, A1, B0, B1, ((uint32_t)i * KQ + (uint32_t)(k - 1)) * 2u, clamp_flags(k, la, lb),
                        keys + (size_t)t * G.npix, s_supp);
        }
        }
    } else {
        // fans t = blockIdx.y + j gridDim.y; within a fan, thread item = kb NT + i, up to the
        // fan's longest ray
        for (int t = blockIdx.y; t < G.n_elem; t += gridDim.y) {
        const int kmax = fan_last_quad(G, fan_len, t);
        const int per_fan = ((kmax + KB - 1) / KB) * NT;
        for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < per_fan; item += gridDim.x * blockDim.x) {
            uint32_t ukb, ui;
            udivmod((uint32_t)item, (uint32_t)NT, nt_magic, ukb, ui);
            const int i = (int)ui, kb = (int)ukb;
            const int la = last_vertex(G, ends, t, i), lb = last_vertex(G, ends, t, i + 1);
            const int k0 = kb * KB + 1, k1 = min(k0 + KB - 1, max(la, lb));
            if (k0 > k1) continue;
            unsigned long long* tab = keys + (size_t)t * G.npix;
            Vtx A0 = get_vtx(verts + vidx(G, t, min(k0 - 1, la), i));
            Vtx B0 = get_vtx(verts + vidx(G, t, min(k0 - 1, lb), i + 1));
            for (int k = k0; k <= k1; ++k) {
                const Vtx A1 = get_vtx(verts + vidx(G, t, min(k, la), i));
                const Vtx B1 = get_vtx(verts + vidx(G, t, min(k, lb), i + 1));
                raster_quad(G, A0, A1, B0, B1, ((uint32_t)i * KQ + (uint32_t)(k - 1)) * 2u, clamp_flags(k, la, lb), tab,
                            s_supp);
                A0 = A1;
                B0 = B1;
            }
        }
        }
    }
}

// The table record of entry (t, pix) from its first-arrival key: from the winning
// triangle id in the tag, its vertices and the pixel (X, Y), the barycentric weights
// (bit-identical to the rasteriser's), then Q, L and the KMAH index of the heaviest
// vertex.  Returns false for a hole (no triangle covered the pixel).
__device__ __forceinline__ bool resolve_entry(const GeoDev& G, const Vtx* __restrict__ verts,
                                              const rb_ray_end* __restrict__ ends, unsigned long long key, int t,
                                              const DF& X, const DF& Y, uint32_t kq_magic, rb_cell& rec) {
    const uint32_t KQ = (uint32_t)(G.max_steps + 1);
    const uint2 kv = make_uint2((uint32_t)key, (uint32_t)(key >> 32));   // {tag, tkey}
    if (kv.y == RB_HOLE) return false;
    const uint32_t id = kv.x >> 8;
    const int half = (int)(id & 1u);
    uint32_t qi, qk1;
    udivmod(id >> 1, KQ, kq_magic, qi, qk1);
    // ids come from the rasteriser (i + 1 < n_rays, 1 <= k1 <= max_steps); clamped all the same
    const int i = min((int)qi, G.n_rays - 2), k1 = min((int)qk1 + 1, G.max_steps);
    // the rays' last vertices matter only where the rasteriser flagged a clamp
    int la = G.max_steps, lb = G.max_steps;
    if (kv.x & 3u) {
        la = last_vertex(G, ends, t, i);
        lb = last_vertex(G, ends, t, i + 1);
    }
    // the winning triangle only: T0 = (A0, B0, B1), T1 = (A0, B1, A1); edge vectors,
    // doubled area (rounded reciprocal) and weights as in bary
    const Vtx A0 = get_vtx(verts + vidx(G, t, min(k1 - 1, la), i));
    const Vtx Vb = get_vtx(half ? verts + vidx(G, t, min(k1, lb), i + 1) : verts + vidx(G, t, min(k1 - 1, lb), i + 1));
    const Vtx Vc = get_vtx(half ? verts + vidx(G, t, min(k1, la), i) : verts + vidx(G, t, min(k1, lb), i + 1));
    const float ux = rel(Vb.xh, Vb.xl, A0.xh, A0.xl), uy = rel(Vb.yh, Vb.yl, A0.yh, A0.yl);
    const float vx = rel(Vc.xh, Vc.xl, A0.xh, A0.xl), vy = rel(Vc.yh, Vc.yl, A0.yh, A0.yl);
    const float ar = __fsub_rn(__fmul_rn(ux, vy), __fmul_rn(uy, vx));
    const float inv = ar != 0.f ? __frcp_rn(ar) : 0.f;
    const float dx = rel(X.hi, X.lo, A0.xh, A0.xl), dy = rel(Y.hi, Y.lo, A0.yh, A0.yl);
    float wa, wb, wc;
    bary(ux, uy, vx, vy, inv, dx, dy, wa, wb, wc);
    int kap = A0.k;
    float wbest = wa;
    if (wb > wbest) { kap = Vb.k; wbest = wb; }
    if (wc > wbest) kap = Vc.k;
    rec.tag = (id << 8) | (uint32_t)min(kap, 255);
    rec.tkey = kv.y;
    rec.q = interp(wa, wb, wc, A0.q, Vb.q, Vc.q);
    rec.l = interp(wa, wb, wc, A0.l, Vb.l, Vc.l);
    return true;
}

// Completes every table record (plain path) from the keys.  Holes stay all ones.
// Thread = pixel (its coordinates and support test computed once), looping over the
// elements t = blockIdx.y, blockIdx.y + gridDim.y, ...; consecutive threads take
// consecutive pixels, so every key load and record store is coalesced.
__global__ void __launch_bounds__(256) k_resolve(GeoDev G, const Vtx* __restrict__ verts,
                                                 const rb_ray_end* __restrict__ ends,
                                                 const unsigned long long* __restrict__ keys, rb_cell* __restrict__ tables,
                                                 uint32_t* __restrict__ counters, uint32_t kq_magic) {
    uint32_t holes = 0;   // support pixels that no triangle of the fan covered
    for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < G.npix; pix += gridDim.x * blockDim.x) {
        const int iy = pix / G.nx, ix = pix - iy * G.nx;
        const DF X = df_pixel_coord(ix, G.cxg, G.h_hi, G.h_lo);
        const DF Y = df_pixel_coord(iy, G.cyg, G.h_hi, G.h_lo);
        const long long jx = 2LL * ix - (G.nx - 1), jy = 2LL * iy - (G.ny - 1);
        const bool in_support = jx * jx + jy * jy <= G.r2max;
        for (int t = blockIdx.y; t < G.n_elem; t += gridDim.y) {
            const size_t u = (size_t)t * G.npix + pix;
            rb_cell rec;
            if (!resolve_entry(G, verts, ends, keys[u], t, X, Y, kq_magic, rec)) {
                rec.tag = RB_HOLE;
                rec.tkey = RB_HOLE;
                rec.q = __uint_as_float(RB_HOLE);
                rec.l = __uint_as_float(RB_HOLE);
                if (in_support) ++holes;
            }
            tables[u] = rec;
        }
    }
    for (int o = 16; o > 0; o >>= 1) holes += __shfl_down_sync(0xffffffffu, holes, o);
    if ((threadIdx.x & 31) == 0 && holes) atomicAdd(counters + CNT_HOLES, holes);
}

// Mixed path: the resolve pass fused with the synthesis of the operand images, so the
// per-(element, pixel) record never goes to memory.  CTA (tile of RB_TP pixels,
// element block of 16), element block major: CTAs side by side take neighbouring tiles
// of the same 16 fans, whose vertex gathers then meet in L2.  Thread (p, half) loads
// the keys of elements 16 eb + 8 half + k (k < 8) at pixel p of the tile, then, four
// elements at a time, resolves them, keeps their synthesis records in registers and
// writes for every frequency of the set the Green's functions of Eqs. 4-5 into row
// 4 eb + 2 half + kg of the pixel's core row in both bf16 planes (the same values as
// the separate record and image passes: the same record, the same formulas).  Four
// records at a time keep the kernel at 64 registers, four CTAs per SM, to hide the
// latency of the vertex gathers.
__global__ void __launch_bounds__(256) k_resolve_images(GeoDev G, const Vtx* __restrict__ verts,
                                                        const rb_ray_end* __restrict__ ends,
                                                        const unsigned long long* __restrict__ keys,
                                                        const float* __restrict__ c, FreqSet F,
                                                        __nv_bfloat16* __restrict__ aimg, size_t a_stride,
                                                        uint32_t* __restrict__ counters, uint32_t kq_magic) {
    const int n = G.n_elem, rcn = 2 * n / 8;
    const int ntiles = (G.npix + RB_TP - 1) / RB_TP;
    const int tile = (int)blockIdx.x % ntiles, eb = (int)blockIdx.x / ntiles;
    const int p = (int)threadIdx.x & (RB_TP - 1), half = (int)threadIdx.x >> 7;
    const int pix = tile * RB_TP + p;
    const int e0 = 16 * eb + 8 * half;
    uint32_t holes = 0;
    const bool live = pix < G.npix;
    const int iy = live ? pix / G.nx : 0, ix = live ? pix - iy * G.nx : 0;
    const DF X = df_pixel_coord(ix, G.cxg, G.h_hi, G.h_lo);
    const DF Y = df_pixel_coord(iy, G.cyg, G.h_hi, G.h_lo);
    const long long jx = 2LL * ix - (G.nx - 1), jy = 2LL * iy - (G.ny - 1);
    const bool in_support = live && jx * jx + jy * jy <= G.r2max;
    const float c_px = live ? __ldg(c + pix) : 0.f;
    unsigned long long key[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) key[k] = live ? keys[(size_t)(e0 + k) * G.npix + pix] : ~0ull;
    // two groups of four elements: one image row (16 bytes per plane) each
#pragma unroll
    for (int kg = 0; kg < 2; ++kg) {
        float4 sr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = e0 + 4 * kg + q;
            rb_cell rec;
            if (!resolve_entry(G, verts, ends, key[4 * kg + q], e, X, Y, kq_magic, rec)) {
                sr[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (in_support) ++holes;
                continue;
            }
            DF ex, ey;
            elem_pos(G, e, ex, ey);
            sr[q] = synth_record(rec, c_px, pixel_elem_dist(G, ix, iy, ex, ey), G.inv_cref, G.inv_cref_lo, G.j_floor);
        }
        for (int fw = 0; fw < F.n; ++fw) {
            __nv_bfloat16* plane = aimg + (size_t)fw * a_stride + (size_t)tile * 2 * rcn * 1024;
            float2 g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q] = green_srec(sr[q], F.f[fw]);
            aimg_put4(plane, rcn, 4 * eb + 2 * half + kg, p, g);
        }
    }
    for (int o = 16; o > 0; o >>= 1) holes += __shfl_down_sync(0xffffffffu, holes, o);
    if ((threadIdx.x & 31) == 0 && holes) atomicAdd(counters + CNT_HOLES, holes);
}

// All-ones fill of the first-arrival keys with one CTA per SM, grid-stride, 16-byte
// stores.  Run on a side stream beside the tracer: a CTA this small co-resides with the
// tracer's CTAs instead of taking their slots, as a full-width fill does.
__global__ void __launch_bounds__(256) k_keys_reset(uint4* K, size_t n16) {
    const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        K[i] = ones;
}

}  // namespace

cudaError_t launch_keys_reset(const GeoDev& G, void* keys, cudaStream_t s) {
    const size_t bytes = (size_t)G.n_elem * G.npix * sizeof(unsigned long long);
    if (((uintptr_t)keys & 15) || (bytes & 15)) return cudaMemsetAsync(keys, 0xff, bytes, s);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 148;
    k_keys_reset<<<nsm, 256, 0, s>>>((uint4*)keys, bytes / 16);
    return cudaGetLastError();
}

cudaError_t launch_trace(const GeoDev& G, const float4* cells, rb_ray_end* ends, const rb_rays* samples,
                         void* keys, rb_cell* tables, void* verts, const float* c, uint32_t* counters,
                         cudaStream_t s, cudaEvent_t traced, cudaEvent_t keys_ready, const FreqSet* F, void* images,
                         int raster_mode, uint32_t* fan_len) {
    rb_rays S{};
    int ws = 0;
    if (samples && samples->vx) {
        S = *samples;
        ws = 1;
    }
    // vertices are stored whenever a buffer is given; gridding needs them and the keys
    const bool grid = keys != nullptr;
    Vtx* V = (Vtx*)verts;
    if (grid && !fan_len) return cudaErrorInvalidValue;
    const bool fused = images != nullptr;
    if (fused && (!F || F->n < 1 || !c || (G.n_elem % 16) != 0)) return cudaErrorInvalidValue;
    if (grid && (!V || (!tables && !fused))) return cudaErrorInvalidValue;
    unsigned long long* K = (unsigned long long*)keys;
    if (grid && !keys_ready) {
        cudaError_t e = cudaMemsetAsync(K, 0xff, (size_t)G.n_elem * G.npix * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    if (grid) {
        cudaError_t e = cudaMemsetAsync(fan_len, 0, (size_t)G.n_elem * sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
    }
    // threads: every fan's rays padded to a multiple of TRACE_GR (the padding returns at once)
    const long long rays = (long long)G.n_elem * ((G.n_rays + TRACE_GR - 1) / TRACE_GR) * TRACE_GR;
    k_trace<<<(int)((rays + 127) / 128), 128, 0, s>>>(G, cells, ends, S, ws, V, counters, grid ? fan_len : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && traced) e = cudaEventRecord(traced, s);   // the end records are complete
    if (e != cudaSuccess || !grid) return e;
    if (keys_ready && (e = cudaStreamWaitEvent(s, keys_ready, 0)) != cudaSuccess) return e;   // keys reset elsewhere
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 148;
    // fans in flight (grid rows): up to 128, fewer where their keys would pass 256 MB, at
    // least 16 (measured on a 256-element ring, 512^2 pixels: 16 fans 1.27 ms, 64 1.23,
    // 128 1.22, 256 1.26)
    int ry = 128;
    while (ry > 16 && (size_t)ry * G.npix * sizeof(unsigned long long) > ((size_t)256 << 20)) ry >>= 1;
    if (ry > G.n_elem) ry = G.n_elem;
    // tube width in pixels where the fan is widest (across the ring): the ray spacing
    // 2 R pi / n_rays over h
    const double tube_px = 2.0 * G.R_d * RB_PI_D / (double)G.n_rays / G.h_d;
    const uint32_t ntm = (uint32_t)(0x100000000ull / (uint32_t)(G.n_rays - 1));
    const size_t ssm = (size_t)G.ny * sizeof(short2);
    const bool along = raster_mode == 1 || (raster_mode == 0 && tube_px >= RASTER_ALONG_K_MIN_PX);
    if (along)
        k_raster<true><<<dim3(nsm * 16 * (256 / raster_threads<true>()) / ry, ry), raster_threads<true>(), ssm, s>>>(G, V, ends, K, fan_len, ntm);
    else
        k_raster<false><<<dim3(nsm * 16 * (256 / raster_threads<false>()) / ry, ry), raster_threads<false>(), ssm, s>>>(G, V, ends, K, fan_len, ntm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint32_t KQ = (uint32_t)(G.max_steps + 1);
    const uint32_t kq_magic = (uint32_t)(0x100000000ull / KQ);
    if (fused) {
        const long long blocks = (long long)((G.npix + RB_TP - 1) / RB_TP) * (G.n_elem / 16);
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        k_resolve_images<<<(int)blocks, 256, 0, s>>>(G, V, ends, K, c, *F, (__nv_bfloat16*)images,
                                                     tc_aimage_elems(G.n_elem, G.npix), counters, kq_magic);
        return cudaGetLastError();
    }
    int bx = (G.npix + 255) / 256;
    int by = 1;
    while (by < 16 && by * 2 <= G.n_elem && (long long)bx * by < (long long)nsm * 16) by *= 2;
    k_resolve<<<dim3(bx, by), 256, 0, s>>>(G, V, ends, K, tables, counters, kq_magic);
    return cudaGetLastError();
}

size_t rb_verts_bytes(int n_elem, int n_rays, int max_steps) {
    return (size_t)n_elem * (size_t)(max_steps + 1) * (size_t)n_rays * sizeof(Vtx);
}
