// Time-of-flight initial guess (Sec. 4: a few linearisations of a ToF reconstruction
// that fits measured times of flight with times of flight along rays).
//
// One linearisation is one SIRT step in slowness s = 1/c along the current rays:
//   ds = D_col^-1 L^T D_row^-1 dT,   dT[e][r] = T_obs - T(c) on the rows used,
// where row (e, r) of L is (1 - lam) times the path of ray i plus lam times the
// path of ray i + 1 of its first-arrival link (the linked time interpolates the two
// rays' times with the same weights), a path integral is the sum over the ray's
// vertex-to-vertex segments of the segment length times the bilinear interpolant at
// the segment midpoint, D_row are the row sums (interpolated path lengths) and D_col
// the column sums.  The per-row mean slowness error dT / D_row is clamped to
// +-2e-3 s/m; rows: receivers on the opposite ~75 % of the ring, linked both in
// the data and in the current medium.  c <- 1 / (1/c + ds) on the support where
// D_col > 0.
//
// Kernels: k_tof_len (path length per ray), k_tof_coef (per fan: each ray's total
// weight sum_r w and weighted error sum_r w dT / D_row, gathered in a fixed order),
// k_tof_bp (per ray: the two coefficients spread along its segments into pixel sums;
// 64-bit fixed-point atomics, so the sums do not depend on the order of arrival),
// k_tof_apply, and k_tof_resid / k_tof_rms for the RMS ToF misfit.
#include "rb_internal.cuh"

namespace {

constexpr float TOF_A_MAX = 2e-3f;    // clamp of the per-row mean slowness error [s/m]
constexpr double FX_ONE = 1099511627776.0;   // 2^40: the largest single deposit in fixed point
constexpr int RT = 256;
constexpr int RB = 256;

__device__ __forceinline__ bool row_used(int e, int r, int N, int gap) {
    int d = e > r ? e - r : r - e;
    d = min(d, N - d);
    return d >= gap;
}

__device__ __forceinline__ float fp_diff(float vh, float vl, float oh, float ol) {
    return __fadd_rn(__fsub_rn(vh, oh), __fsub_rn(vl, ol));
}

__device__ __forceinline__ Vtx load_vtx(const Vtx* __restrict__ p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    return Vtx{a.x, a.y, a.z, a.w, b.x, b.y, b.z, __float_as_int(b.w)};
}

// path length of every ray: the sum of its vertex-to-vertex segment lengths
__global__ void __launch_bounds__(128) k_tof_len(GeoDev G, const Vtx* __restrict__ verts,
                                                 const rb_ray_end* __restrict__ ends, float* __restrict__ len) {
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long long)G.n_elem * G.n_rays) return;
    const int t = (int)(ray / G.n_rays), i = (int)(ray % G.n_rays);
    const int nv = ends[ray].n_vert;
    double acc = 0.0;
    if (nv > 1) {
        Vtx a = load_vtx(verts + vtx_index(G, t, 0, i));
        for (int k = 1; k < nv; ++k) {
            const Vtx b = load_vtx(verts + vtx_index(G, t, k, i));
            const float dx = fp_diff(b.xh, b.xl, a.xh, a.xl), dy = fp_diff(b.yh, b.yl, a.yh, a.yl);
            acc += (double)sqrtf(dx * dx + dy * dy);
            a = b;
        }
    }
    len[ray] = (float)acc;
}

// Per fan e: the rows' mean slowness errors, then per ray i the weighted error a_i and the
// total weight b_i of the rows that use it (receivers scanned in index order); the largest
// |a| and b (as float bits, an order-independent maximum) set the fixed-point scales.
__global__ void __launch_bounds__(RT) k_tof_coef(GeoDev G, const LinkRec* __restrict__ lrec,
                                                 const double* __restrict__ t_obs, const uint8_t* __restrict__ obs_linked,
                                                 const float* __restrict__ len, float2* __restrict__ coef,
                                                 uint32_t* __restrict__ amax) {
    extern __shared__ unsigned char smem[];
    const int N = G.n_elem, n = G.n_rays, e = blockIdx.x;
    int* sb = (int*)smem;                   // [N] winning interval (-1: row not used)
    float* sl = (float*)(sb + N);           // [N] lam
    float* se = sl + N;                     // [N] mean slowness error
    const int gap = (N + 7) / 8;
    for (int r = threadIdx.x; r < N; r += RT) {
        const size_t o = (size_t)e * N + r;
        const LinkRec L = lrec[o];
        int b = -1;
        float lam = 0.f, err = 0.f;
        if (L.i >= 0 && obs_linked[o] && row_used(e, r, N, gap)) {
            lam = L.lam;
            const double drow = (1.0 - (double)lam) * (double)len[(size_t)e * n + L.i] +
                                (double)lam * (double)len[(size_t)e * n + L.i + 1];
            if (drow > 0.0) {
                b = L.i;
                const double m = (t_obs[o] - L.T) / drow;
                err = fminf(fmaxf((float)m, -TOF_A_MAX), TOF_A_MAX);
            }
        }
        sb[r] = b;
        sl[r] = lam;
        se[r] = err;
    }
    __syncthreads();
    float am = 0.f, bm = 0.f;
    for (int i = threadIdx.x; i < n; i += RT) {
        float a = 0.f, w = 0.f;
        for (int r = 0; r < N; ++r) {
            const int b = sb[r];
            if (b == i) {
                a = fmaf(1.f - sl[r], se[r], a);
                w += 1.f - sl[r];
            } else if (b == i - 1) {
                a = fmaf(sl[r], se[r], a);
                w += sl[r];
            }
        }
        coef[(size_t)e * n + i] = make_float2(a, w);
        am = fmaxf(am, fabsf(a));
        bm = fmaxf(bm, w);
    }
    if (am > 0.f) atomicMax(&amax[0], __float_as_uint(am));
    if (bm > 0.f) atomicMax(&amax[1], __float_as_uint(bm));
}

__device__ __forceinline__ void deposit(unsigned long long* __restrict__ dst, double v) {
    const long long q = __double2ll_rn(v);
    if (q != 0) atomicAdd(dst, (unsigned long long)q);
}

// Per ray: a_i and b_i spread along the ray's segments into the pixel sums, in fixed
// point (one unit = the largest |a| (or b) times ds, over 2^40).  Consecutive segments
// with the same bilinear quad are merged before the atomics.
__global__ void __launch_bounds__(128) k_tof_bp(GeoDev G, const Vtx* __restrict__ verts,
                                                const rb_ray_end* __restrict__ ends, const float2* __restrict__ coef,
                                                const uint32_t* __restrict__ amax, unsigned long long* __restrict__ num,
                                                unsigned long long* __restrict__ den) {
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long long)G.n_elem * G.n_rays) return;
    const float2 cf = coef[ray];
    const int nv = ends[ray].n_vert;
    if (nv < 2 || (cf.x == 0.f && cf.y == 0.f)) return;
    const int t = (int)(ray / G.n_rays), i = (int)(ray % G.n_rays);
    const float am = __uint_as_float(amax[0]), bm = __uint_as_float(amax[1]);
    const double sa = am > 0.f ? FX_ONE / ((double)am * G.ds_d) : 0.0;
    const double sb = bm > 0.f ? FX_ONE / ((double)bm * G.ds_d) : 0.0;
    int q00 = -1;
    double w4[4] = {0.0, 0.0, 0.0, 0.0};
    auto flush = [&]() {
        if (q00 < 0) return;
        const int px[4] = {q00, q00 + 1, q00 + G.nx, q00 + G.nx + 1};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            deposit(num + px[j], (double)cf.x * w4[j] * sa);
            deposit(den + px[j], (double)cf.y * w4[j] * sb);
            w4[j] = 0.0;
        }
    };
    Vtx a = load_vtx(verts + vtx_index(G, t, 0, i));
    for (int k = 1; k < nv; ++k) {
        const Vtx b = load_vtx(verts + vtx_index(G, t, k, i));
        const float dx = fp_diff(b.xh, b.xl, a.xh, a.xl), dy = fp_diff(b.yh, b.yl, a.yh, a.yl);
        const float l = sqrtf(dx * dx + dy * dy);
        const float mx = (a.xh + a.xl) + 0.5f * dx, my = (a.yh + a.yl) + 0.5f * dy;
        const float u = fminf(fmaxf(fmaf(mx, G.inv_h, G.cxg), 0.f), (float)(G.nx - 1));
        const float v = fminf(fmaxf(fmaf(my, G.inv_h, G.cyg), 0.f), (float)(G.ny - 1));
        const int i0 = min((int)u, G.nx - 2), j0 = min((int)v, G.ny - 2);
        const float fu = u - (float)i0, fv = v - (float)j0;
        const int q = j0 * G.nx + i0;
        if (q != q00) {
            flush();
            q00 = q;
        }
        w4[0] += (double)((1.f - fu) * (1.f - fv) * l);
        w4[1] += (double)(fu * (1.f - fv) * l);
        w4[2] += (double)((1.f - fu) * fv * l);
        w4[3] += (double)(fu * fv * l);
        a = b;
    }
    flush();
}

__device__ __forceinline__ bool in_support_px(const GeoDev& G, int pix) {
    const int ix = pix % G.nx, iy = pix / G.nx;
    const long long jx = 2LL * ix - (G.nx - 1), jy = 2LL * iy - (G.ny - 1);
    return jx * jx + jy * jy <= G.r2max;
}

__global__ void __launch_bounds__(RT) k_tof_apply(GeoDev G, float* __restrict__ c, const unsigned long long* __restrict__ num,
                                                  const unsigned long long* __restrict__ den,
                                                  const uint32_t* __restrict__ amax) {
    const float am = __uint_as_float(amax[0]), bm = __uint_as_float(amax[1]);
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += gridDim.x * RT) {
        const long long dq = (long long)den[p];
        if (dq <= 0 || !in_support_px(G, p)) continue;
        // num / den back in physical units: (nq am ds / 2^40) / (dq bm ds / 2^40)
        const double ds = ((double)(long long)num[p] * (double)am) / ((double)dq * (double)bm);
        c[p] = (float)(1.0 / (1.0 / (double)c[p] + ds));
    }
}

// partial sums of dT^2 and of the row count over the rows used
__global__ void __launch_bounds__(RT) k_tof_resid(GeoDev G, const LinkRec* __restrict__ lrec,
                                                  const double* __restrict__ t_obs,
                                                  const uint8_t* __restrict__ obs_linked, double* __restrict__ part) {
    const int N = G.n_elem, gap = (N + 7) / 8;
    double s2 = 0.0, cnt = 0.0;
    for (long long o = (long long)blockIdx.x * RT + threadIdx.x; o < (long long)N * N; o += (long long)RB * RT) {
        const int e = (int)(o / N), r = (int)(o % N);
        const LinkRec L = lrec[o];
        if (L.i >= 0 && obs_linked[o] && row_used(e, r, N, gap)) {
            const double d = t_obs[o] - L.T;
            s2 += d * d;
            cnt += 1.0;
        }
    }
    __shared__ double a[RT], b[RT];
    a[threadIdx.x] = s2;
    b[threadIdx.x] = cnt;
    __syncthreads();
    for (int k = RT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            a[threadIdx.x] += a[threadIdx.x + k];
            b[threadIdx.x] += b[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a[0];
        part[RB + blockIdx.x] = b[0];
    }
}

__global__ void __launch_bounds__(RT) k_tof_rms(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double a[RT], b[RT];
    a[threadIdx.x] = part[threadIdx.x];
    b[threadIdx.x] = part[RB + threadIdx.x];
    __syncthreads();
    for (int k = RT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            a[threadIdx.x] += a[threadIdx.x + k];
            b[threadIdx.x] += b[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = b[0] > 0.0 ? sqrt(a[0] / b[0]) : 0.0;
}

__global__ void __launch_bounds__(RT) k_tof_times_out(int n2, const LinkRec* __restrict__ lrec, double* __restrict__ t_out) {
    for (int o = blockIdx.x * RT + threadIdx.x; o < n2; o += gridDim.x * RT) t_out[o] = lrec[o].i >= 0 ? lrec[o].T : 0.0;
}

}  // namespace

size_t tof_ws_bytes(int n_elem, int n_rays, int npix) {
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return al((size_t)n_elem * n_elem * sizeof(LinkRec)) + al((size_t)n_elem * n_rays * 4) +
           al((size_t)n_elem * n_rays * 8) + 2 * al((size_t)npix * 8) + 256;
}

namespace {
struct TofWs {
    LinkRec* lrec;
    float* len;
    float2* coef;
    unsigned long long* num;
    unsigned long long* den;
    uint32_t* amax;
};
TofWs carve(const GeoDev& G, void* base) {
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char* p = (char*)base;
    TofWs w;
    w.lrec = (LinkRec*)p;
    p += al((size_t)G.n_elem * G.n_elem * sizeof(LinkRec));
    w.len = (float*)p;
    p += al((size_t)G.n_elem * G.n_rays * 4);
    w.coef = (float2*)p;
    p += al((size_t)G.n_elem * G.n_rays * 8);
    w.num = (unsigned long long*)p;
    p += al((size_t)G.npix * 8);
    w.den = (unsigned long long*)p;
    p += al((size_t)G.npix * 8);
    w.amax = (uint32_t*)p;
    return w;
}
}  // namespace

cudaError_t launch_tof_link(const GeoDev& G, const float* c, const rb_ray_end* ends, void* tof_ws, uint8_t* linked,
                            cudaStream_t s) {
    FreqSet F;
    F.n = 0;
    return launch_link(G, c, ends, F, nullptr, linked, s, carve(G, tof_ws).lrec);
}

cudaError_t launch_tof_times_out(const GeoDev& G, void* tof_ws, double* t_out, cudaStream_t s) {
    k_tof_times_out<<<RB, RT, 0, s>>>(G.n_elem * G.n_elem, carve(G, tof_ws).lrec, t_out);
    return cudaGetLastError();
}

cudaError_t launch_tof_resid(const GeoDev& G, void* tof_ws, const double* t_obs, const uint8_t* obs_linked,
                             double* part, double* out, cudaStream_t s) {
    k_tof_resid<<<RB, RT, 0, s>>>(G, carve(G, tof_ws).lrec, t_obs, obs_linked, part);
    k_tof_rms<<<1, RT, 0, s>>>(part, out);
    return cudaGetLastError();
}

// one SIRT step on the current rays (vertices in verts, links in the ToF workspace)
cudaError_t launch_tof_step(const GeoDev& G, const Vtx* verts, const rb_ray_end* ends, void* tof_ws, const double* t_obs,
                            const uint8_t* obs_linked, float* c, cudaStream_t s) {
    const TofWs w = carve(G, tof_ws);
    const long long rays = (long long)G.n_elem * G.n_rays;
    const int rb = (int)((rays + 127) / 128);
    k_tof_len<<<rb, 128, 0, s>>>(G, verts, ends, w.len);
    cudaError_t e = cudaMemsetAsync(w.num, 0, (size_t)((char*)w.amax - (char*)w.num) + 8, s);
    if (e != cudaSuccess) return e;
    const size_t sm = (size_t)G.n_elem * 12;
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(k_tof_coef, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_tof_coef<<<G.n_elem, RT, sm, s>>>(G, w.lrec, t_obs, obs_linked, w.len, w.coef, w.amax);
    k_tof_bp<<<rb, 128, 0, s>>>(G, verts, ends, w.coef, w.amax, w.num, w.den);
    k_tof_apply<<<RB, RT, 0, s>>>(G, c, w.num, w.den, w.amax);
    return cudaGetLastError();
}
