/*
 * FP64 CPU oracle for the ray part of the ray-Born forward model: ray fans
 * (Eikonal and Transport equations, Eqs. 6-7) and their gridding onto pixels.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  It shares no code with the CUDA library and
 * is called only by the tests, the smoke check and the CPU-baseline timing.
 *
 * Every step follows the definitions written out in oracle/rays.py and
 * oracle/grid.py (which call into this file):
 *   - fields c, c_x, c_y, c_xx, c_xy, c_yy, alpha0 are sampled by bilinear
 *     interpolation of their pixel-centre grids (clamped at the grid edge);
 *   - each ray integrates, in arclength s with classical RK4 and fixed step ds,
 *       x' = cos th, y' = sin th, th' = (c_x sin th - c_y cos th)/c,
 *       T' = 1/c,  Q' = c P,  P' = -(c_nn/c^2) Q,  L' = alpha0,
 *     with c_nn = c_xx sin^2 th - 2 c_xy sin th cos th + c_yy cos^2 th.
 *     The first equations are the characteristics of the Eikonal equation
 *     (Eq. 6, phase = omega T); Q, P are dynamic ray tracing, whose Q is the
 *     ray-tube width that solves the Transport equation (Eq. 7).
 *   - a ray stops at the first step k >= 1 with |x_k| >= R; its last vertex is
 *     the crossing of the segment x_{k-1} x_k with the ring, every state
 *     component interpolated linearly at the crossing.
 *   - gridding splits each quad of neighbouring rays into two triangles,
 *     interpolates linearly with barycentric weights and keeps the first
 *     arrival (smallest interpolated traveltime) per pixel.
 * Plain loops, double precision throughout; OpenMP only over independent fans.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 9  /* per-vertex record: x, y, th, T, Q, P, L, kappa, s */
enum { VX = 0, VY, VTH, VT, VQ, VP, VL, VK, VS };

typedef struct {
    int32_t n_elem;
    double ring_radius;
    int32_t nx, ny;
    double h;
    int32_t n_rays;
    double ds;
    int32_t max_steps;
    double support_margin;
    double c_ref;
} orc_geom;

typedef struct { double x, y, th, T, Q, P, L; } orc_state;

/* bilinear interpolation of the 7 field grids F[7][ny][nx] at (x, y) */
static void bilinear(const orc_geom* g, const double* F, double x, double y, double out[7]) {
    const int nx = g->nx, ny = g->ny;
    double u = x / g->h + 0.5 * (nx - 1);
    double v = y / g->h + 0.5 * (ny - 1);
    if (u < 0.0) u = 0.0;
    if (u > nx - 1) u = nx - 1;
    if (v < 0.0) v = 0.0;
    if (v > ny - 1) v = ny - 1;
    int i0 = (int)floor(u), j0 = (int)floor(v);
    if (i0 > nx - 2) i0 = nx - 2;
    if (j0 > ny - 2) j0 = ny - 2;
    double fu = u - i0, fv = v - j0;
    const size_t plane = (size_t)nx * ny;
    for (int f = 0; f < 7; ++f) {
        const double* P = F + f * plane;
        double v00 = P[(size_t)j0 * nx + i0], v10 = P[(size_t)j0 * nx + i0 + 1];
        double v01 = P[(size_t)(j0 + 1) * nx + i0], v11 = P[(size_t)(j0 + 1) * nx + i0 + 1];
        out[f] = (1 - fu) * (1 - fv) * v00 + fu * (1 - fv) * v10 + (1 - fu) * fv * v01 + fu * fv * v11;
    }
}

static void deriv(const orc_geom* g, const double* F, const orc_state* s, orc_state* d) {
    double f[7];
    bilinear(g, F, s->x, s->y, f);
    const double c = f[0], cx = f[1], cy = f[2], cxx = f[3], cxy = f[4], cyy = f[5], a0 = f[6];
    const double sn = sin(s->th), cs = cos(s->th);
    const double cnn = cxx * sn * sn - 2.0 * cxy * sn * cs + cyy * cs * cs;
    d->x = cs;
    d->y = sn;
    d->th = (cx * sn - cy * cs) / c;
    d->T = 1.0 / c;
    d->Q = c * s->P;
    d->P = -(cnn / (c * c)) * s->Q;
    d->L = a0;
}

static void axpy(orc_state* out, const orc_state* s, double a, const orc_state* k) {
    out->x = s->x + a * k->x;
    out->y = s->y + a * k->y;
    out->th = s->th + a * k->th;
    out->T = s->T + a * k->T;
    out->Q = s->Q + a * k->Q;
    out->P = s->P + a * k->P;
    out->L = s->L + a * k->L;
}

static void rk4(const orc_geom* g, const double* F, const orc_state* s, orc_state* o) {
    const double ds = g->ds;
    orc_state k1, k2, k3, k4, t;
    deriv(g, F, s, &k1);
    axpy(&t, s, 0.5 * ds, &k1);
    deriv(g, F, &t, &k2);
    axpy(&t, s, 0.5 * ds, &k2);
    deriv(g, F, &t, &k3);
    axpy(&t, s, ds, &k3);
    deriv(g, F, &t, &k4);
    const double w = ds / 6.0;
    o->x = s->x + w * (k1.x + 2.0 * k2.x + 2.0 * k3.x + k4.x);
    o->y = s->y + w * (k1.y + 2.0 * k2.y + 2.0 * k3.y + k4.y);
    o->th = s->th + w * (k1.th + 2.0 * k2.th + 2.0 * k3.th + k4.th);
    o->T = s->T + w * (k1.T + 2.0 * k2.T + 2.0 * k3.T + k4.T);
    o->Q = s->Q + w * (k1.Q + 2.0 * k2.Q + 2.0 * k3.Q + k4.Q);
    o->P = s->P + w * (k1.P + 2.0 * k2.P + 2.0 * k3.P + k4.P);
    o->L = s->L + w * (k1.L + 2.0 * k2.L + 2.0 * k3.L + k4.L);
}

static void put(double* V, const orc_state* s, double kappa, double arclen) {
    V[VX] = s->x; V[VY] = s->y; V[VTH] = s->th; V[VT] = s->T;
    V[VQ] = s->Q; V[VP] = s->P; V[VL] = s->L; V[VK] = kappa; V[VS] = arclen;
}

/* parameter in [0,1] where the segment a -> b leaves the circle |x| = R */
static double exit_lambda(double ax, double ay, double bx, double by, double R) {
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
    if (lam < 0.0) lam = 0.0;
    if (lam > 1.0) lam = 1.0;
    return lam;
}

static int signbit_d(double v) { return signbit(v) ? 1 : 0; }

/*
 * Trace ray i of the fan of element t.  Writes vertices V[0..n-1] (NV doubles
 * each) and returns n, the vertex count including the exit point.  *lost is
 * set when the ray did not reach the ring within max_steps (then all
 * max_steps+1 integrated states are returned as vertices).
 */
static int trace_ray(const orc_geom* g, const double* F, int t, int i, double* V, int* lost) {
    const double pi = 3.14159265358979323846;
    const double phi = 2.0 * pi * t / g->n_elem;
    const double R = g->ring_radius;
    const double psi = -0.5 * pi + (i + 0.5) * pi / g->n_rays;
    orc_state s;
    s.x = R * cos(phi);
    s.y = R * sin(phi);
    s.th = phi + pi + psi;
    double f[7];
    bilinear(g, F, s.x, s.y, f);
    s.T = 0.0; s.Q = 0.0; s.P = 1.0 / f[0]; s.L = 0.0;
    double kappa = 0.0;
    put(V, &s, kappa, 0.0);
    *lost = 0;
    for (int k = 1; k <= g->max_steps; ++k) {
        orc_state n;
        rk4(g, F, &s, &n);
        if (n.x * n.x + n.y * n.y >= R * R) {
            const double lam = exit_lambda(s.x, s.y, n.x, n.y, R);
            orc_state e;
            e.x = s.x + lam * (n.x - s.x);
            e.y = s.y + lam * (n.y - s.y);
            e.th = s.th + lam * (n.th - s.th);
            e.T = s.T + lam * (n.T - s.T);
            e.Q = s.Q + lam * (n.Q - s.Q);
            e.P = s.P + lam * (n.P - s.P);
            e.L = s.L + lam * (n.L - s.L);
            double ke = kappa + ((k >= 2 && signbit_d(e.Q) != signbit_d(s.Q)) ? 1.0 : 0.0);
            put(V + (size_t)k * NV, &e, ke, (k - 1 + lam) * g->ds);
            return k + 1;
        }
        if (k >= 2 && signbit_d(n.Q) != signbit_d(s.Q)) kappa += 1.0;
        put(V + (size_t)k * NV, &n, kappa, k * g->ds);
        s = n;
    }
    *lost = 1;
    return g->max_steps + 1;
}

/* One fan: all rays' vertices, V[n_rays][max_steps+1][NV], nvert[n_rays]. Returns lost-ray count. */
int orc_trace_fan(const orc_geom* g, const double* F, int t, double* V, int32_t* nvert) {
    int nlost = 0;
    const size_t stride = (size_t)(g->max_steps + 1) * NV;
    for (int i = 0; i < g->n_rays; ++i) {
        int lost;
        nvert[i] = trace_ray(g, F, t, i, V + i * stride, &lost);
        nlost += lost;
    }
    return nlost;
}

/* All fans, last vertex of every ray: E[n_elem][n_rays][NV]; nvert[n_elem][n_rays]; lost[n_elem][n_rays]. */
int orc_trace_endpoints(const orc_geom* g, const double* F, double* E, int32_t* nvert, int32_t* lost) {
    const size_t stride = (size_t)(g->max_steps + 1) * NV;
    int total = 0;
#pragma omp parallel reduction(+ : total)
    {
        double* V = (double*)malloc(stride * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int64_t tr = 0; tr < (int64_t)g->n_elem * g->n_rays; ++tr) {
            const int t = (int)(tr / g->n_rays), i = (int)(tr % g->n_rays);
            int l;
            const int n = trace_ray(g, F, t, i, V, &l);
            nvert[tr] = n;
            lost[tr] = l;
            total += l;
            memcpy(E + tr * NV, V + (size_t)(n - 1) * NV, NV * sizeof(double));
        }
        free(V);
    }
    return total;
}

/*
 * Grid one fan onto the pixels of the support.  Output per pixel p (OUT[p][6]):
 *   T_res  = sum_j w_j (T_j - |v_j - x_t| / c_ref)  (traveltime minus the
 *            straight water time, interpolated; the gridded traveltime is
 *            |p - x_t| / c_ref + T_res),
 *   Q, L   = sum_j w_j Q_j, sum_j w_j L_j,
 *   kappa  = KMAH count of the vertex with the largest weight,
 *   tri    = winning triangle id ((i * (max_steps+1) + k) * 2 + half),
 *   hit    = 1 if covered, 0 for a hole.
 * The winner is the triangle with the smallest interpolated T_res (the
 * first arrival); ties keep the earliest triangle id.
 */
#define NO 6
static void grid_fan(const orc_geom* g, int t, const double* V, const int32_t* nvert, int64_t r2max,
                     double* OUT) {
    const double pi = 3.14159265358979323846;
    const double phi = 2.0 * pi * t / g->n_elem;
    const double xt = g->ring_radius * cos(phi), yt = g->ring_radius * sin(phi);
    const int nx = g->nx, ny = g->ny;
    const double h = g->h;
    const double X0 = -0.5 * (nx - 1) * h, Y0 = -0.5 * (ny - 1) * h;
    const size_t stride = (size_t)(g->max_steps + 1) * NV;
    const int KQ = g->max_steps + 1;
    for (size_t p = 0; p < (size_t)nx * ny; ++p) {
        OUT[p * NO + 0] = INFINITY;
        OUT[p * NO + 1] = 0; OUT[p * NO + 2] = 0; OUT[p * NO + 3] = 0;
        OUT[p * NO + 4] = -1; OUT[p * NO + 5] = 0;
    }
    for (int i = 0; i + 1 < g->n_rays; ++i) {
        const int na = nvert[i], nb = nvert[i + 1];
        const int nq = (na > nb ? na : nb) - 1;
        const double* Va = V + (size_t)i * stride;
        const double* Vb = V + (size_t)(i + 1) * stride;
        for (int k = 0; k < nq; ++k) {
            const double* A0 = Va + (size_t)(k < na - 1 ? k : na - 1) * NV;
            const double* A1 = Va + (size_t)(k + 1 < na - 1 ? k + 1 : na - 1) * NV;
            const double* B0 = Vb + (size_t)(k < nb - 1 ? k : nb - 1) * NV;
            const double* B1 = Vb + (size_t)(k + 1 < nb - 1 ? k + 1 : nb - 1) * NV;
            for (int half = 0; half < 2; ++half) {
                const double* P[3];
                if (half == 0) { P[0] = A0; P[1] = B0; P[2] = B1; }
                else           { P[0] = A0; P[1] = B1; P[2] = A1; }
                const double ax = P[0][VX], ay = P[0][VY];
                const double bx = P[1][VX], by = P[1][VY];
                const double cx = P[2][VX], cy = P[2][VY];
                const double area2 = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
                if (area2 == 0.0) continue;
                double tr[3];
                for (int q = 0; q < 3; ++q) {
                    const double dx = P[q][VX] - xt, dy = P[q][VY] - yt;
                    tr[q] = P[q][VT] - sqrt(dx * dx + dy * dy) / g->c_ref;
                }
                double xmin = fmin(ax, fmin(bx, cx)), xmax = fmax(ax, fmax(bx, cx));
                double ymin = fmin(ay, fmin(by, cy)), ymax = fmax(ay, fmax(by, cy));
                int ix0 = (int)floor((xmin - X0) / h), ix1 = (int)ceil((xmax - X0) / h);
                int iy0 = (int)floor((ymin - Y0) / h), iy1 = (int)ceil((ymax - Y0) / h);
                if (ix0 < 0) ix0 = 0;
                if (iy0 < 0) iy0 = 0;
                if (ix1 > nx - 1) ix1 = nx - 1;
                if (iy1 > ny - 1) iy1 = ny - 1;
                const double tri_id = (double)(((int64_t)i * KQ + k) * 2 + half);
                for (int iy = iy0; iy <= iy1; ++iy) {
                    const int64_t jy = 2 * (int64_t)iy - (ny - 1);
                    for (int ix = ix0; ix <= ix1; ++ix) {
                        const int64_t jx = 2 * (int64_t)ix - (nx - 1);
                        if (jx * jx + jy * jy > r2max) continue;
                        const double px = X0 + ix * h, py = Y0 + iy * h;
                        const double wb = ((px - ax) * (cy - ay) - (py - ay) * (cx - ax)) / area2;
                        const double wc = ((bx - ax) * (py - ay) - (by - ay) * (px - ax)) / area2;
                        const double wa = 1.0 - wb - wc;
                        if (wa < -1e-12 || wb < -1e-12 || wc < -1e-12) continue;
                        const double trp = wa * tr[0] + wb * tr[1] + wc * tr[2];
                        double* o = OUT + ((size_t)iy * nx + ix) * NO;
                        if (!(trp < o[0])) continue;
                        o[0] = trp;
                        o[1] = wa * P[0][VQ] + wb * P[1][VQ] + wc * P[2][VQ];
                        o[2] = wa * P[0][VL] + wb * P[1][VL] + wc * P[2][VL];
                        int best = 0;
                        if (wb > wa) best = 1;
                        if (wc > (best == 0 ? wa : wb)) best = 2;
                        o[3] = P[best][VK];
                        o[4] = tri_id;
                        o[5] = 1.0;
                    }
                }
            }
        }
    }
    for (size_t p = 0; p < (size_t)nx * ny; ++p)
        if (OUT[p * NO + 5] == 0.0) OUT[p * NO + 0] = 0.0;
}

/* All fans: OUT[n_elem][nx*ny][NO]. r2max: pixel (ix,iy) is in the support iff
 * (2ix-(nx-1))^2 + (2iy-(ny-1))^2 <= r2max.  Returns the lost-ray count. */
int orc_grid(const orc_geom* g, const double* F, int64_t r2max, double* OUT) {
    const size_t stride = (size_t)(g->max_steps + 1) * NV;
    const size_t npix = (size_t)g->nx * g->ny;
    int total = 0;
#pragma omp parallel reduction(+ : total)
    {
        double* V = (double*)malloc(stride * g->n_rays * sizeof(double));
        int32_t* nvert = (int32_t*)malloc(sizeof(int32_t) * g->n_rays);
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < g->n_elem; ++t) {
            total += orc_trace_fan(g, F, t, V, nvert);
            grid_fan(g, t, V, nvert, r2max, OUT + (size_t)t * npix * NO);
        }
        free(V);
        free(nvert);
    }
    return total;
}

/* All fans, but only the listed pixels are kept: OUT[n_elem][n_sel][NO]. */
int orc_grid_pixels(const orc_geom* g, const double* F, int64_t r2max, const int64_t* sel, int64_t n_sel,
                    double* OUT) {
    const size_t stride = (size_t)(g->max_steps + 1) * NV;
    const size_t npix = (size_t)g->nx * g->ny;
    int total = 0;
#pragma omp parallel reduction(+ : total)
    {
        double* V = (double*)malloc(stride * g->n_rays * sizeof(double));
        int32_t* nvert = (int32_t*)malloc(sizeof(int32_t) * g->n_rays);
        double* full = (double*)malloc(npix * NO * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < g->n_elem; ++t) {
            total += orc_trace_fan(g, F, t, V, nvert);
            grid_fan(g, t, V, nvert, r2max, full);
            for (int64_t j = 0; j < n_sel; ++j)
                memcpy(OUT + ((size_t)t * n_sel + j) * NO, full + (size_t)sel[j] * NO, NO * sizeof(double));
        }
        free(V);
        free(nvert);
        free(full);
    }
    return total;
}
