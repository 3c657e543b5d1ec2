// Field preparation: element positions and the cell-packed derivative grids
// that the ray integrator samples.
//
// The Eikonal characteristics (Eq. 6) need c and grad c along a ray and the
// dynamic ray tracing that solves the Transport equation (Eq. 7) needs the
// Hessian of c.  Discretisation: first derivatives by central differences
// over index-clamped neighbours (one-sided at the grid edge); second
// derivatives c_xx, c_yy by the three-point stencil centred at the nearest
// interior pixel; c_xy by the mixed central difference over clamped
// neighbours.  Each grid is sampled by bilinear interpolation.
//
// Layout: one 128-byte record per grid cell (i0, j0), i0 < nx-1, j0 < ny-1,
// holding for each of c, c_x, c_y, c_xx, c_xy, c_yy, alpha0 the coefficients
// (a, b, c, d) of its bilinear interpolant a + b u + c v + d u v over the cell
// (u, v in [0, 1]), from the corner values q00 = (i0, j0), q10, q01, q11:
// a = q00, b = q10 - q00, c = q01 - q00, d = q11 - q10 - q01 + q00.  The fields go
// in pairs (c, c_x), (c_y, c_xx), (c_xy, c_yy), two float4 per pair:
// {a_F, a_G, b_F, b_G}, {c_F, c_G, d_F, d_G}, so that the sampler evaluates a pair
// with packed two-lane FMAs; then alpha0's {a, b, c, d} and a pad.  A ray that enters
// a cell loads one aligned 128-byte line and keeps it in registers until it leaves
// the cell.
#include "rb_internal.cuh"

__global__ void k_elem_positions(GeoDev G, float4* xy) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G.n_elem) return;
    double phi = 2.0 * RB_PI_D * (double)t / (double)G.n_elem;
    double s, c;
    sincos(phi, &s, &c);
    const DF x = df_from_double(G.R_d * c), y = df_from_double(G.R_d * s);
    xy[t] = make_float4(x.hi, x.lo, y.hi, y.lo);
}

cudaError_t launch_elem_positions(const GeoDev& G, float4* elem_xy, cudaStream_t s) {
    k_elem_positions<<<(G.n_elem + 127) / 128, 128, 0, s>>>(G, elem_xy);
    return cudaGetLastError();
}

struct PixF { float c, cx, cy, cxx, cxy, cyy; };

__device__ __forceinline__ PixF pixel_fields(const float* __restrict__ c, int nx, int ny, float h, int ix, int iy) {
    const int ip = min(ix + 1, nx - 1), im = max(ix - 1, 0);
    const int jp = min(iy + 1, ny - 1), jm = max(iy - 1, 0);
    const int ic = min(max(ix, 1), nx - 2), jc = min(max(iy, 1), ny - 2);
    auto C = [&](int i, int j) { return __ldg(c + (size_t)j * nx + i); };
    const float dxs = (float)(ip - im) * h, dys = (float)(jp - jm) * h;
    const float ih2 = 1.0f / (h * h);
    PixF f;
    f.c = C(ix, iy);
    f.cx = (C(ip, iy) - C(im, iy)) / dxs;
    f.cy = (C(ix, jp) - C(ix, jm)) / dys;
    f.cxx = (C(ic + 1, iy) - 2.0f * C(ic, iy) + C(ic - 1, iy)) * ih2;
    f.cyy = (C(ix, jc + 1) - 2.0f * C(ix, jc) + C(ix, jc - 1)) * ih2;
    f.cxy = ((C(ip, jp) - C(ip, jm)) - (C(im, jp) - C(im, jm))) / (dxs * dys);
    return f;
}

__global__ void k_fields(GeoDev G, const float* __restrict__ c, const float* __restrict__ a0, float4* __restrict__ cells) {
    const int ncx = G.nx - 1, ncy = G.ny - 1;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncx * ncy) return;
    const int i0 = cell % ncx, j0 = cell / ncx;
    PixF q[4];
    float a[4];
    const int ci[4] = {i0, i0 + 1, i0, i0 + 1};
    const int cj[4] = {j0, j0, j0 + 1, j0 + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        q[k] = pixel_fields(c, G.nx, G.ny, G.h, ci[k], cj[k]);
        a[k] = __ldg(a0 + (size_t)cj[k] * G.nx + ci[k]);
    }
    float4* o = cells + (size_t)cell * 8;
    auto coef = [](float q00, float q10, float q01, float q11) {
        return make_float4(q00, q10 - q00, q01 - q00, (q11 - q10) - (q01 - q00));
    };
    auto pair = [&](float4* dst, float4 f, float4 g) {
        dst[0] = make_float4(f.x, g.x, f.y, g.y);
        dst[1] = make_float4(f.z, g.z, f.w, g.w);
    };
    pair(o + 0, coef(q[0].c, q[1].c, q[2].c, q[3].c), coef(q[0].cx, q[1].cx, q[2].cx, q[3].cx));
    pair(o + 2, coef(q[0].cy, q[1].cy, q[2].cy, q[3].cy), coef(q[0].cxx, q[1].cxx, q[2].cxx, q[3].cxx));
    pair(o + 4, coef(q[0].cxy, q[1].cxy, q[2].cxy, q[3].cxy), coef(q[0].cyy, q[1].cyy, q[2].cyy, q[3].cyy));
    o[6] = coef(a[0], a[1], a[2], a[3]);
    o[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_fields(const GeoDev& G, const float* c, const float* alpha0, float4* cells, cudaStream_t s) {
    const int n = (G.nx - 1) * (G.ny - 1);
    k_fields<<<(n + 255) / 256, 256, 0, s>>>(G, c, alpha0, cells);
    return cudaGetLastError();
}
