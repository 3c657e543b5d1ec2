// One-step update (the diagonal-Hessian solve of Eq. 10, Sec. 3).
//
//   eps   = eps_rel * mean over the support of sum_w H_w
//   p(x)  = -sum_w Re g_w(x) / (sum_w H_w(x) + eps)   on the support, 0 outside
//   alpha = -<sum_w Re g_w, p> / sum_w sum_{e,r} W |B_w p|^2   (RB_STEP_EXACT; 1 for RB_STEP_DIAG)
//   dm    = alpha p,  dc = -dm c^3 / (2 h^2),  c <- c + dc,  ||dc||_2 over the support.
//
// Every reduction is two-level with a fixed shape: a fixed grid writes one
// double partial per block (fixed thread-to-element map, tree inside the
// block) and a single block sums the partials in a fixed tree, so results do
// not depend on scheduling.  All scalars stay on the device.
#include "rb_internal.cuh"

namespace {

constexpr int RB = 256;   // reduction blocks
constexpr int RT = 256;   // threads per reduction block

__device__ __forceinline__ bool in_support(const GeoDev& G, int pix) {
    const int ix = pix % G.nx, iy = pix / G.nx;
    const long long jx = 2LL * ix - (G.nx - 1), jy = 2LL * iy - (G.ny - 1);
    return jx * jx + jy * jy <= G.r2max;
}

__device__ __forceinline__ void block_sum_store(double v, double* dst) {
    __shared__ double s[RT];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int k = RT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *dst = s[0];
}

// phase 0: partial sums of hsum over the support, and the support size
__global__ void __launch_bounds__(RT) k_hsum_part(GeoDev G, const float* __restrict__ hsum, double* __restrict__ part) {
    double acc = 0.0, cnt = 0.0;
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += RB * RT)
        if (in_support(G, p)) {
            acc += (double)hsum[p];
            cnt += 1.0;
        }
    block_sum_store(acc, part + blockIdx.x);
    __syncthreads();
    block_sum_store(cnt, part + RB + blockIdx.x);
}

__global__ void __launch_bounds__(RT) k_eps(const double* __restrict__ part, double eps_rel, double* __restrict__ dbl) {
    __shared__ double s[RT], t[RT];
    s[threadIdx.x] = part[threadIdx.x];
    t[threadIdx.x] = part[RB + threadIdx.x];
    __syncthreads();
    for (int k = RT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            s[threadIdx.x] += s[threadIdx.x + k];
            t[threadIdx.x] += t[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dbl[DBL_HMEAN] = t[0] > 0.0 ? s[0] / t[0] : 0.0;
        dbl[DBL_EPS] = eps_rel * dbl[DBL_HMEAN];
    }
}

// single-block fixed-order sum of n partials:  dst[slot] = (accumulate ? dst[slot] : 0) + scale * sum
__global__ void __launch_bounds__(RT) k_sum_part(const double* __restrict__ part, int n, double* __restrict__ dbl, int slot,
                                                 double scale, int accumulate) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += RT) acc += part[i];
    __shared__ double s[RT];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = RT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) dbl[slot] = (accumulate ? dbl[slot] : 0.0) + scale * s[0];
}

// phase 1: direction p and partials of -<g, p>
__global__ void __launch_bounds__(RT) k_direction(GeoDev G, const float* __restrict__ gsum, const float* __restrict__ hsum,
                                                  const double* __restrict__ dbl, float* __restrict__ pdir,
                                                  double* __restrict__ part) {
    const float eps = (float)dbl[DBL_EPS];
    double acc = 0.0;
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += RB * RT) {
        float v = 0.f;
        if (in_support(G, p)) {
            const float gv = gsum[p];
            v = -gv / (hsum[p] + eps);
            acc -= (double)v * (double)gv;
        }
        pdir[p] = v;
    }
    block_sum_store(acc, part + blockIdx.x);
}

// phase 2: alpha, dc, c update and partials of ||dc||^2
__global__ void __launch_bounds__(RT) k_apply(GeoDev G, float* __restrict__ c, const float* __restrict__ pdir,
                                              double* __restrict__ dbl, int step_mode, float* __restrict__ dc_out,
                                              double* __restrict__ part) {
    double alpha = 1.0;
    if (step_mode == RB_STEP_EXACT) {
        const double den = dbl[DBL_DEN];
        alpha = den > 0.0 ? dbl[DBL_NUM] / den : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) dbl[DBL_ALPHA] = alpha;
    const float af = (float)alpha;
    const float s = 1.0f / (2.0f * G.h * G.h);
    double acc = 0.0;
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += RB * RT) {
        const float cv = c[p];
        const float dm = af * pdir[p];
        const float dc = -dm * cv * cv * cv * s;
        if (dc_out) dc_out[p] = dc;
        c[p] = cv + dc;
        if (in_support(G, p)) acc += (double)dc * (double)dc;
    }
    block_sum_store(acc, part + blockIdx.x);
}

// ---------------------------------------------------------------------------
// CG variant: preconditioned conjugate gradients (Hestenes and Stiefel, 1952) on the
// normal equations of the linearised objective of Eq. 10,
//   A dm = b,  A = sum_w Re(B_w^H W B_w),  b = -sum_w Re g_w,  over the support, dm_0 = 0.
// M^-1 = 1/(sum_w H_w + eps) per pixel (precond), or the scalar 1/(mean H + eps): a scalar
// preconditioner leaves the CG iterates those of plain CG and keeps A p within FP32 range.
// The curvature <p_k, A p_k> is taken as sum_w sum_{e,r} W |B_w p_k|^2 from the forward
// reduction (equal in exact arithmetic, non-negative by construction).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cg_minv(const float* __restrict__ hsum, int p, int precond, float eps, float hm) {
    return precond ? 1.0f / (hsum[p] + eps) : 1.0f / (hm + eps);
}

__global__ void __launch_bounds__(RT) k_cg_init(GeoDev G, const float* __restrict__ gsum, const float* __restrict__ hsum,
                                                const double* __restrict__ dbl, int precond, float* __restrict__ x,
                                                float* __restrict__ r, float* __restrict__ pv, double* __restrict__ part) {
    const float eps = (float)dbl[DBL_EPS], hm = (float)dbl[DBL_HMEAN];
    double acc = 0.0;
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += RB * RT) {
        float rv = 0.f, zv = 0.f;
        if (in_support(G, p)) {
            rv = -gsum[p];
            zv = cg_minv(hsum, p, precond, eps, hm) * rv;
            acc += (double)rv * (double)zv;
        }
        x[p] = 0.f;
        r[p] = rv;
        pv[p] = zv;
    }
    block_sum_store(acc, part + blockIdx.x);
}

// x += alpha p, r -= alpha q (alpha = rho_k / <p_k, A p_k>, 0 when the curvature is not
// positive); partials of rho_{k+1} = <r, M^-1 r>
__global__ void __launch_bounds__(RT) k_cg_xr(GeoDev G, const float* __restrict__ hsum, const double* __restrict__ dbl,
                                              int precond, int k, float* __restrict__ x, float* __restrict__ r,
                                              const float* __restrict__ pv, const float* __restrict__ q,
                                              double* __restrict__ part) {
    const float eps = (float)dbl[DBL_EPS], hm = (float)dbl[DBL_HMEAN];
    const double pap = dbl[DBL_CG_PAP + k];
    const float a = pap > 0.0 ? (float)(dbl[DBL_CG_RHO + k] / pap) : 0.f;
    double acc = 0.0;
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += RB * RT) {
        if (!in_support(G, p)) continue;
        x[p] = fmaf(a, pv[p], x[p]);
        const float rv = fmaf(-a, q[p], r[p]);
        r[p] = rv;
        acc += (double)rv * (double)(cg_minv(hsum, p, precond, eps, hm) * rv);
    }
    block_sum_store(acc, part + blockIdx.x);
}

// p = M^-1 r + beta p,  beta = rho_{k+1} / rho_k
__global__ void __launch_bounds__(RT) k_cg_p(GeoDev G, const float* __restrict__ hsum, const double* __restrict__ dbl,
                                             int precond, int k, const float* __restrict__ r, float* __restrict__ pv) {
    const float eps = (float)dbl[DBL_EPS], hm = (float)dbl[DBL_HMEAN];
    const double rho = dbl[DBL_CG_RHO + k];
    const float beta = rho != 0.0 ? (float)(dbl[DBL_CG_RHO + k + 1] / rho) : 0.f;
    for (int p = blockIdx.x * RT + threadIdx.x; p < G.npix; p += RB * RT)
        if (in_support(G, p)) pv[p] = fmaf(beta, pv[p], cg_minv(hsum, p, precond, eps, hm) * r[p]);
}

// The diagnostics record (when asked for), and the lost-ray count into the caller
// stream's host-mapped limit word when rays were lost (read by the next update call).
__global__ void k_finish(const double* __restrict__ dbl, const uint32_t* __restrict__ cnt, rb_diag* __restrict__ diag,
                         uint32_t* __restrict__ limit_word) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (limit_word && cnt[CNT_LOST] > 0) *(volatile uint32_t*)limit_word = cnt[CNT_LOST];
    if (!diag) return;
    rb_diag d;
    d.dc_norm = sqrt(dbl[DBL_NORM2]);
    d.alpha = dbl[DBL_ALPHA];
    d.eps = dbl[DBL_EPS];
    d.lost_rays = cnt[CNT_LOST];
    d.holes = cnt[CNT_HOLES];
    d.unlinked = cnt[CNT_UNLINKED];
    d.kept = cnt[CNT_KEPT];
    d.zeroed = cnt[CNT_ZEROED];
    d.tc_timeouts = cnt[CNT_TC_TIMEOUT];
    *diag = d;
}

}  // namespace

// Launch sequence pieces used by rb_hf_update (rb_api.cu).
cudaError_t launch_update(const GeoDev& G, float* c, const float* gsum, const float* hsum, float* pdir, float* dc_out,
                          double* part, double* dbl, uint32_t* counters, rb_diag* diag, double eps_rel, int step_mode,
                          int phase, cudaStream_t s, uint32_t* limit_word) {
    switch (phase) {
        case 0: {  // eps, direction, numerator
            k_hsum_part<<<RB, RT, 0, s>>>(G, hsum, part);
            k_eps<<<1, RT, 0, s>>>(part, eps_rel, dbl);
            k_direction<<<RB, RT, 0, s>>>(G, gsum, hsum, dbl, pdir, part);
            k_sum_part<<<1, RT, 0, s>>>(part, RB, dbl, DBL_NUM, 1.0, 0);
            break;
        }
        case 1: {  // apply the step and finish
            k_apply<<<RB, RT, 0, s>>>(G, c, pdir, dbl, step_mode, dc_out, part);
            k_sum_part<<<1, RT, 0, s>>>(part, RB, dbl, DBL_NORM2, 1.0, 0);
            if (diag || limit_word) k_finish<<<1, 32, 0, s>>>(dbl, counters, diag, limit_word);
            break;
        }
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cg_init(const GeoDev& G, const float* gsum, const float* hsum, int precond, float* x, float* r,
                           float* p, double* part, double* dbl, double eps_rel, cudaStream_t s) {
    k_hsum_part<<<RB, RT, 0, s>>>(G, hsum, part);
    k_eps<<<1, RT, 0, s>>>(part, eps_rel, dbl);
    k_cg_init<<<RB, RT, 0, s>>>(G, gsum, hsum, dbl, precond, x, r, p, part);
    k_sum_part<<<1, RT, 0, s>>>(part, RB, dbl, DBL_CG_RHO, 1.0, 0);
    return cudaGetLastError();
}

// after <p_k, A p_k> is in DBL_CG_PAP + k: x, r, rho_{k+1}, then p_{k+1}
cudaError_t launch_cg_step(const GeoDev& G, const float* hsum, int precond, int k, float* x, float* r, float* p,
                           const float* q, double* part, double* dbl, cudaStream_t s) {
    k_cg_xr<<<RB, RT, 0, s>>>(G, hsum, dbl, precond, k, x, r, p, q, part);
    k_sum_part<<<1, RT, 0, s>>>(part, RB, dbl, DBL_CG_RHO + k + 1, 1.0, 0);
    k_cg_p<<<RB, RT, 0, s>>>(G, hsum, dbl, precond, k, r, p);
    return cudaGetLastError();
}

__global__ void k_cg_history(const double* __restrict__ dbl, int iters, double* __restrict__ hist) {
    const int k = threadIdx.x;
    const double rho0 = dbl[DBL_CG_RHO];
    if (k <= iters) hist[k] = rho0 != 0.0 ? dbl[DBL_CG_RHO + k] / rho0 : 0.0;
}

cudaError_t launch_cg_history(const double* dbl, int iters, double* hist, cudaStream_t s) {
    k_cg_history<<<1, 32, 0, s>>>(dbl, iters, hist);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* part, int n, double* dbl, int slot, double scale, int accumulate,
                                cudaStream_t s) {
    k_sum_part<<<1, RT, 0, s>>>(part, n, dbl, slot, scale, accumulate);
    return cudaGetLastError();
}
