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
// triangle id), resolved by a 128-bit compare-and-swap on the table record.
//
// GB300 mapping: one warp owns 32 consecutive rays of one fan (31 tubes;
// neighbouring warps overlap by one ray, which both trace bit-identically),
// so a tube's four vertices are two registers and one shuffle away and the
// ray samples never reach HBM.  Field samples come from the 128-byte cell
// records of rb_fields.cu, kept in registers while a ray stays in its cell.
// Positions and the direction are float pairs (compensated sums); the
// traveltime is integrated as the residual T - |x - x_t|/c_ref in double,
// which keeps the Green's-function phase w T accurate at MHz frequencies.
#include "rb_internal.cuh"

namespace {

struct Cache {
    int id;
    float4 c, cx, cy, cxx, cxy, cyy, a0;
};

struct Deriv { float x, y, th, t, q, p, l; };

struct Vtx { float xh, xl, yh, yl, t, q, l; int k; };

__device__ __forceinline__ void sample(const GeoDev& G, const float4* __restrict__ cells, Cache& cc, float px, float py,
                                       float f[7]) {
    float u = fminf(fmaxf(fmaf(px, G.inv_h, G.cxg), 0.f), (float)(G.nx - 1));
    float v = fminf(fmaxf(fmaf(py, G.inv_h, G.cyg), 0.f), (float)(G.ny - 1));
    const int i0 = min((int)u, G.nx - 2), j0 = min((int)v, G.ny - 2);
    const float fu = u - (float)i0, fv = v - (float)j0;
    const int id = j0 * (G.nx - 1) + i0;
    if (id != cc.id) {
        const float4* p = cells + (size_t)id * 8;
        cc.c = __ldg(p + 0);
        cc.cx = __ldg(p + 1);
        cc.cy = __ldg(p + 2);
        cc.cxx = __ldg(p + 3);
        cc.cxy = __ldg(p + 4);
        cc.cyy = __ldg(p + 5);
        cc.a0 = __ldg(p + 6);
        cc.id = id;
    }
    const float w00 = (1.f - fu) * (1.f - fv), w10 = fu * (1.f - fv), w01 = (1.f - fu) * fv, w11 = fu * fv;
#define RB_BL(q) (w00 * (q).x + w10 * (q).y + w01 * (q).z + w11 * (q).w)
    f[0] = RB_BL(cc.c);
    f[1] = RB_BL(cc.cx);
    f[2] = RB_BL(cc.cy);
    f[3] = RB_BL(cc.cxx);
    f[4] = RB_BL(cc.cxy);
    f[5] = RB_BL(cc.cyy);
    f[6] = RB_BL(cc.a0);
#undef RB_BL
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
        sincosf(th_hi + d, &s, &c);
    }
}

struct RayCtx {
    float xs_hi, xs_lo, ys_hi, ys_lo;  // source position
};

__device__ __forceinline__ Deriv eval_stage(const GeoDev& G, const float4* __restrict__ cells, Cache& cc,
                                            float xh, float xl, float yh, float yl, float rxh, float rxl, float ryh,
                                            float ryl, float C0, float S0, float thh, float thl, float q, float p,
                                            float a, const Deriv& kp) {
    const float ox = fmaf(a, kp.x, xl), oy = fmaf(a, kp.y, yl);
    const float px = xh + ox, py = yh + oy;
    const float rx = rxh + fmaf(a, kp.x, rxl), ry = ryh + fmaf(a, kp.y, ryl);
    float cth, sth;
    rotate(C0, S0, thh, fmaf(a, kp.th, thl), cth, sth);
    const float qs = fmaf(a, kp.q, q), ps = fmaf(a, kp.p, p);
    float f[7];
    sample(G, cells, cc, px, py, f);
    const float c = f[0];
    const float rc = 1.0f / c;
    Deriv d;
    d.x = cth;
    d.y = sth;
    d.th = (f[1] * sth - f[2] * cth) * rc;
    // T_res' = 1/c - (t . r_hat)/c_ref = (c_ref - c)/(c c_ref) + (1 - t . r_hat)/c_ref,
    // with 1 - t.r_hat = (t x r)^2 / (|r| (|r| + t.r)) (no cancellation).
    const float rr = sqrtf(rx * rx + ry * ry);
    float one_m_cos = 0.f;
    if (rr > 0.f) {
        const float dot = cth * rx + sth * ry;
        const float crs = cth * ry - sth * rx;
        const float den = rr * (rr + dot);
        one_m_cos = den > 0.f ? (crs * crs) / den : 2.f;
    }
    d.t = (G.c_ref - c) * (rc * G.inv_cref) + one_m_cos * G.inv_cref;
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

// Atomic "keep the smaller (tkey, tag)" on a 16-byte table record.  The first
// attempt assumes the record is still a hole (all bytes 0xff), which is the common
// case, so no load precedes it; a failed attempt returns the current record.
__device__ __forceinline__ void cell_min(rb_cell* dst, uint32_t tkey, uint32_t tag, float q, float l,
                                        uint32_t* giveup) {
    const unsigned long long nk = ((unsigned long long)tkey << 32) | tag;
    const unsigned long long nv = ((unsigned long long)__float_as_uint(l) << 32) | __float_as_uint(q);
    unsigned long long ck = ~0ull, cv = ~0ull;
    int it = 0;
    for (; it < 256; ++it) {
        unsigned long long ok, ov;
        asm volatile(
            "{\n\t.reg .b128 d, cmp, val;\n\t"
            "mov.b128 cmp, {%2, %3};\n\t"
            "mov.b128 val, {%4, %5};\n\t"
            "atom.relaxed.gpu.global.cas.b128 d, [%6], cmp, val;\n\t"
            "mov.b128 {%0, %1}, d;\n\t}"
            : "=l"(ok), "=l"(ov)
            : "l"(ck), "l"(cv), "l"(nk), "l"(nv), "l"(dst)
            : "memory");
        if (ok == ck && ov == cv) break;   // stored
        ck = ok;
        cv = ov;
        if (!(nk < ck)) break;             // an earlier arrival (or tie winner) is already there
    }
    if (it == 256) atomicAdd(giveup, 1u);
}

// Rasterise one ray-tube quad: triangles T0 = (A0, B0, B1) (id base) and
// T1 = (A0, B1, A1) (id base + 1), A = this ray, B = the next ray, 0/1 = steps k-1/k.
// One pixel box (pixel centres inside the quad's bounding box) serves both
// triangles; where both contain a pixel the smaller T_res (then T0) is kept.
// Coordinates are taken relative to A0 from float-pair differences.
__device__ __forceinline__ void raster_quad(const GeoDev& G, const Vtx& A0, const Vtx& A1, const Vtx& B0, const Vtx& B1,
                                            uint32_t base, rb_cell* __restrict__ tab, uint32_t* giveup) {
    const float b0x = (B0.xh - A0.xh) + (B0.xl - A0.xl), b0y = (B0.yh - A0.yh) + (B0.yl - A0.yl);
    const float b1x = (B1.xh - A0.xh) + (B1.xl - A0.xl), b1y = (B1.yh - A0.yh) + (B1.yl - A0.yl);
    const float a1x = (A1.xh - A0.xh) + (A1.xl - A0.xl), a1y = (A1.yh - A0.yh) + (A1.yl - A0.yl);
    // twice the signed areas; exactly zero when two vertices coincide (frozen or shared vertices)
    const float ar0 = __fsub_rn(__fmul_rn(b0x, b1y), __fmul_rn(b0y, b1x));
    const float ar1 = __fsub_rn(__fmul_rn(b1x, a1y), __fmul_rn(b1y, a1x));
    const bool t0 = ar0 != 0.f, t1 = ar1 != 0.f;
    if (!t0 && !t1) return;
    const float i0 = t0 ? 1.0f / ar0 : 0.f, i1 = t1 ? 1.0f / ar1 : 0.f;
    // tight box of pixel centres (index space), with a 1e-3 px guard
    const float ua = fmaf(A0.xh, G.inv_h, G.cxg) + A0.xl * G.inv_h;
    const float va = fmaf(A0.yh, G.inv_h, G.cyg) + A0.yl * G.inv_h;
    const float xmin = fminf(fminf(0.f, b0x), fminf(b1x, a1x)), xmax = fmaxf(fmaxf(0.f, b0x), fmaxf(b1x, a1x));
    const float ymin = fminf(fminf(0.f, b0y), fminf(b1y, a1y)), ymax = fmaxf(fmaxf(0.f, b0y), fmaxf(b1y, a1y));
    const int ix0 = max(0, (int)ceilf(fmaf(xmin, G.inv_h, ua) - 1e-3f));
    const int ix1 = min(G.nx - 1, (int)floorf(fmaf(xmax, G.inv_h, ua) + 1e-3f));
    const int iy0 = max(0, (int)ceilf(fmaf(ymin, G.inv_h, va) - 1e-3f));
    const int iy1 = min(G.ny - 1, (int)floorf(fmaf(ymax, G.inv_h, va) + 1e-3f));
    const float tol = -1e-6f;
    for (int iy = iy0; iy <= iy1; ++iy) {
        const long long jy = 2LL * iy - (G.ny - 1);
        const DF Y = df_pixel_coord(iy, G.cyg, G.h_hi, G.h_lo);
        const float dy = (Y.hi - A0.yh) + (Y.lo - A0.yl);
        for (int ix = ix0; ix <= ix1; ++ix) {
            const long long jx = 2LL * ix - (G.nx - 1);
            if (jx * jx + jy * jy > G.r2max) continue;
            const DF X = df_pixel_coord(ix, G.cxg, G.h_hi, G.h_lo);
            const float dx = (X.hi - A0.xh) + (X.lo - A0.xl);
            bool in0 = false, in1 = false;
            float wb0 = 0.f, wc0 = 0.f, wa0 = 0.f, wb1 = 0.f, wc1 = 0.f, wa1 = 0.f;
            if (t0) {
                wb0 = (dx * b1y - dy * b1x) * i0;
                wc0 = (b0x * dy - b0y * dx) * i0;
                wa0 = 1.f - wb0 - wc0;
                in0 = wa0 >= tol && wb0 >= tol && wc0 >= tol;
            }
            if (t1) {
                wb1 = (dx * a1y - dy * a1x) * i1;
                wc1 = (b1x * dy - b1y * dx) * i1;
                wa1 = 1.f - wb1 - wc1;
                in1 = wa1 >= tol && wb1 >= tol && wc1 >= tol;
            }
            if (!in0 && !in1) continue;
            const float tr0 = in0 ? wa0 * A0.t + wb0 * B0.t + wc0 * B1.t : 0.f;
            const float tr1 = in1 ? wa1 * A0.t + wb1 * B1.t + wc1 * A1.t : 0.f;
            const bool use1 = in1 && (!in0 || tr1 < tr0);
            float tr, q, l;
            int kap;
            uint32_t id;
            if (!use1) {
                tr = tr0;
                q = wa0 * A0.q + wb0 * B0.q + wc0 * B1.q;
                l = wa0 * A0.l + wb0 * B0.l + wc0 * B1.l;
                kap = A0.k;
                float wbest = wa0;
                if (wb0 > wbest) { kap = B0.k; wbest = wb0; }
                if (wc0 > wbest) kap = B1.k;
                id = base;
            } else {
                tr = tr1;
                q = wa1 * A0.q + wb1 * B1.q + wc1 * A1.q;
                l = wa1 * A0.l + wb1 * B1.l + wc1 * A1.l;
                kap = A0.k;
                float wbest = wa1;
                if (wb1 > wbest) { kap = B1.k; wbest = wb1; }
                if (wc1 > wbest) kap = A1.k;
                id = base + 1u;
            }
            const uint32_t tag = (id << 8) | (uint32_t)min(kap, 255);
            cell_min(tab + (size_t)iy * G.nx + ix, f2key(tr), tag, q, l, giveup);
        }
    }
}

__device__ __forceinline__ Vtx shfl_down_vtx(const Vtx& v) {
    Vtx o;
    o.xh = __shfl_down_sync(0xffffffffu, v.xh, 1);
    o.xl = __shfl_down_sync(0xffffffffu, v.xl, 1);
    o.yh = __shfl_down_sync(0xffffffffu, v.yh, 1);
    o.yl = __shfl_down_sync(0xffffffffu, v.yl, 1);
    o.t = __shfl_down_sync(0xffffffffu, v.t, 1);
    o.q = __shfl_down_sync(0xffffffffu, v.q, 1);
    o.l = __shfl_down_sync(0xffffffffu, v.l, 1);
    o.k = __shfl_down_sync(0xffffffffu, v.k, 1);
    return o;
}

__global__ void __launch_bounds__(128) k_trace(GeoDev G, const float4* __restrict__ cells, rb_ray_end* __restrict__ ends,
                                               rb_rays S, int write_samples, rb_cell* __restrict__ tables,
                                               uint32_t* __restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gw >= G.n_elem * G.n_wpf) return;  // uniform per warp
    const int t = gw / G.n_wpf, wi = gw % G.n_wpf;
    const int i = wi * 31 + lane;
    const bool valid = i < G.n_rays;
    const bool owner = valid && (lane < 31 || i == G.n_rays - 1);
    const bool tube = (lane < 31) && (i + 1 < G.n_rays);
    rb_cell* tab = tables ? tables + (size_t)t * G.npix : nullptr;
    uint32_t* giveup = counters + CNT_CAS_GIVEUP;

    DF xs, ys;
    elem_pos(G, t, xs, ys);
    const double xs_d = (double)xs.hi + (double)xs.lo, ys_d = (double)ys.hi + (double)ys.lo;
    const double th0 = 2.0 * RB_PI_D * (double)t / (double)G.n_elem + 0.5 * RB_PI_D +
                       ((double)i + 0.5) * RB_PI_D / (double)G.n_rays;
    const DF thd = df_from_double(th0);

    Cache cc;
    cc.id = -1;
    float f0[7];
    sample(G, cells, cc, xs.hi + xs.lo, ys.hi + ys.lo, f0);

    float xh = xs.hi, xl = xs.lo, yh = ys.hi, yl = ys.lo, thh = thd.hi, thl = thd.lo;
    double tres = 0.0;
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
    Vtx nb_cur = shfl_down_vtx(cur);
    const uint32_t KQ = (uint32_t)(G.max_steps + 1);
    const float ds = G.ds, a2 = 0.5f * G.ds, ds6 = G.ds * (1.0f / 6.0f);

    for (int k = 1; k <= G.max_steps; ++k) {
        if (!__any_sync(0xffffffffu, alive)) break;
        const Vtx prev = cur, nb_prev = nb_cur;
        if (alive) {
            float C0, S0;
            sincosf(thh, &S0, &C0);
            const float rxh = xh - xs.hi, rxl = xl - xs.lo, ryh = yh - ys.hi, ryl = yl - ys.lo;
            const Deriv z{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const Deriv k1 = eval_stage(G, cells, cc, xh, xl, yh, yl, rxh, rxl, ryh, ryl, C0, S0, thh, thl, q, p, 0.f, z);
            const Deriv k2 = eval_stage(G, cells, cc, xh, xl, yh, yl, rxh, rxl, ryh, ryl, C0, S0, thh, thl, q, p, a2, k1);
            const Deriv k3 = eval_stage(G, cells, cc, xh, xl, yh, yl, rxh, rxl, ryh, ryl, C0, S0, thh, thl, q, p, a2, k2);
            const Deriv k4 = eval_stage(G, cells, cc, xh, xl, yh, yl, rxh, rxl, ryh, ryl, C0, S0, thh, thl, q, p, ds, k3);
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
            const double ntres = tres + (double)it;
            const float nq = q + iq, np = p + ip, nl = l + il;
            // exit test: float screen, then double decision
            const float fx = nxh + nxl, fy = nyh + nyl;
            bool out = false;
            if (fx * fx + fy * fy >= G.R2 * (1.0f - 4e-6f)) {
                const double dx = (double)nxh + (double)nxl, dy = (double)nyh + (double)nyl;
                out = dx * dx + dy * dy >= G.R_d * G.R_d;
            }
            if (out) {
                const double ax = (double)xh + (double)xl, ay = (double)yh + (double)yl;
                const double bx = (double)nxh + (double)nxl, by = (double)nyh + (double)nyl;
                const double lam = exit_lambda(ax, ay, bx, by, G.R_d);
                const float lf = (float)lam;
                const double ex = ax + lam * (bx - ax), ey = ay + lam * (by - ay);
                const double etres = tres + lam * (ntres - tres);
                const double eth = ((double)thh + (double)thl) + lam * (((double)nthh + (double)nthl) - ((double)thh + (double)thl));
                const float eq = q + lf * (nq - q), ep = p + lf * (np - p), el = l + lf * (nl - l);
                const int ek = kap + ((k >= 2 && signbit(eq) != signbit(q)) ? 1 : 0);
                const DF exd = df_from_double(ex), eyd = df_from_double(ey);
                xh = exd.hi; xl = exd.lo; yh = eyd.hi; yl = eyd.lo;
                q = eq; p = ep; l = el; kap = ek; tres = etres;
                alive = false;
                if (owner) {
                    const double ddx = ex - xs_d, ddy = ey - ys_d;
                    rb_ray_end e;
                    e.t_res = etres;
                    e.t = etres + sqrt(ddx * ddx + ddy * ddy) * (1.0 / G.c_ref_d);
                    e.x = ex;
                    e.y = ey;
                    e.theta = (float)eth;
                    e.q = eq;
                    e.p = ep;
                    e.l = el;
                    e.kappa = ek;
                    e.n_vert = k + 1;
                    ends[(size_t)t * G.n_rays + i] = e;
                }
            } else {
                if (k >= 2 && signbit(nq) != signbit(q)) ++kap;
                xh = nxh; xl = nxl; yh = nyh; yl = nyl; thh = nthh; thl = nthl;
                tres = ntres; q = nq; p = np; l = nl;
                if (k == G.max_steps) {
                    alive = false;
                    if (owner) {
                        const double ex = (double)xh + (double)xl, ey = (double)yh + (double)yl;
                        const double ddx = ex - xs_d, ddy = ey - ys_d;
                        rb_ray_end e;
                        e.t_res = tres;
                        e.t = tres + sqrt(ddx * ddx + ddy * ddy) * (1.0 / G.c_ref_d);
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
                    }
                }
            }
            cur = Vtx{xh, xl, yh, yl, (float)tres, q, l, kap};
            if (write_samples) {
                const size_t o = sbase + (size_t)k;
                const double vx = (double)xh + (double)xl, vy = (double)yh + (double)yl;
                const double ddx = vx - xs_d, ddy = vy - ys_d;
                S.vx[o] = (float)vx;
                S.vy[o] = (float)vy;
                S.vt[o] = tres + sqrt(ddx * ddx + ddy * ddy) * (1.0 / G.c_ref_d);
                S.vq[o] = q;
                S.vl[o] = l;
                S.vkappa[o] = kap;
            }
        }
        nb_cur = shfl_down_vtx(cur);
        if (tab && tube) {
            const uint32_t base = ((uint32_t)i * KQ + (uint32_t)(k - 1)) * 2u;
            raster_quad(G, prev, cur, nb_prev, nb_cur, base, tab, giveup);
        }
    }
}

}  // namespace

cudaError_t launch_trace(const GeoDev& G, const float4* cells, rb_ray_end* ends, const rb_rays* samples,
                         rb_cell* tables, uint32_t* counters, cudaStream_t s) {
    rb_rays S{};
    int ws = 0;
    if (samples && samples->vx) {
        S = *samples;
        ws = 1;
    }
    const long long warps = (long long)G.n_elem * G.n_wpf;
    const int blocks = (int)((warps * 32 + 127) / 128);
    k_trace<<<blocks, 128, 0, s>>>(G, cells, ends, S, ws, tables, counters);
    return cudaGetLastError();
}
