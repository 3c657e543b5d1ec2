/*
 * rb.h - C-ABI of the GB300 ray-Born library (librb.so).
 *
 * One Hessian-free ray-Born update of a sound-speed map from ring-array
 * transmission data (arXiv 2511.16633): ray fans through the current sound
 * speed, their traveltime / spreading / absorption gridded into per-pixel
 * Green's functions, the Born forward and adjoint contractions and a
 * diagonal-Hessian one-step update.  Every entry point launches CUDA kernels
 * for sm_103a on the caller's stream.
 *
 * Conventions shared by every call:
 *   - Array arguments are DEVICE pointers unless stated otherwise; the caller
 *     owns them.  Pixels are row-major, flat index iy*nx + ix, pixel (ix, iy)
 *     centred at ((ix - (nx-1)/2) h, (iy - (ny-1)/2) h).  Element t of the
 *     ring sits at angle 2 pi t / n_elem.  Complex values are interleaved
 *     (re, im) float pairs.  Units are SI (m, s, Hz); alpha0 is in
 *     dB / (MHz^y cm).
 *   - The library allocates no device memory, frees nothing and never
 *     synchronises the device: all scratch comes from the caller's workspace,
 *     sized by rb_workspace_size() (rb_born_forward_noalloc excepted, see
 *     there).  Calls are asynchronous and stream-ordered.  rb_hf_update and
 *     rb_cg_update run part of their work on a library stream kept for the
 *     caller's stream on the current device (created with four events on the
 *     first such call from that stream and kept for the process; past 256 such
 *     streams callers share them), forked from and joined back into the
 *     caller's stream inside the call, so their results are ordered on the
 *     caller's stream as usual.
 *   - Argument and shape errors are detected on the host before any launch
 *     and returned synchronously; a failed launch returns RB_ERR_CUDA.
 *     Data-dependent conditions found on the device (a ray that does not
 *     reach the ring within max_steps, uncovered pixels, unlinked pairs) are
 *     counted in an rb_diag record the caller can read afterwards; no kernel
 *     traps and every device loop is bounded.  Lost rays are also reported
 *     without synchronisation: an update that lost rays sets a host-mapped word
 *     kept for its stream, and the next rb_hf_update or rb_cg_update from that
 *     stream and workspace that finds the word set (the lossy update has
 *     completed by then) clears it and returns RB_ERR_LIMIT before launching
 *     anything (a call with another workspace discards the pending report).
 *   - Calls are reentrant given distinct workspaces.  The only global state is
 *     those library streams with their events and limit words (a mutex orders
 *     the host threads that fork and join them), the fixed scratch array of
 *     rb_born_forward_noalloc, and the constant status strings.
 */
#ifndef RB_H
#define RB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (0 = legacy default stream). */
typedef struct CUstream_st* rb_stream;

typedef enum {
    RB_OK = 0,
    RB_ERR_ARG = 1,         /* null pointer, non-positive size, bad enum value */
    RB_ERR_SHAPE = 2,       /* sizes outside the supported ranges */
    RB_ERR_WORKSPACE = 3,   /* workspace missing, too small or misaligned */
    RB_ERR_CUDA = 4,        /* a CUDA launch or call failed */
    RB_ERR_LIMIT = 5,       /* an earlier rb_hf_update / rb_cg_update from the same stream and workspace lost rays
                               (a ray still inside the ring after max_steps): reported once by the next
                               such call that finds it, which then launches nothing */
    RB_ERR_UNSUPPORTED = 6  /* valid request the library does not implement */
} rb_status;

typedef enum {
    RB_PREC_FP32 = 0,       /* plain FP32 CUDA-core contractions (the adjoint, and so rb_born_adjoint,
                               rb_hf_update and rb_cg_update, for rings of up to 512 elements) */
    RB_PREC_BF16X3 = 1      /* tcgen05 BF16 tensor cores, 3-term split products, FP32 accumulation
                               (rings of 64..256 elements in multiples of 64, and of 512, 768
                               and 1024) */
} rb_precision;             /* other ring sizes return RB_ERR_UNSUPPORTED before any work */

typedef enum {
    RB_STEP_EXACT = 0,      /* diagonal-Hessian direction, scaled by the exact line minimum of Eq. 10 */
    RB_STEP_DIAG = 1        /* diagonal-Hessian step alone */
} rb_step_mode;

/* Acquisition, grid and ray-fan parameters (host struct, passed by pointer). */
typedef struct rb_geometry {
    int32_t n_elem;         /* ring elements, each an emitter and a receiver (2..1024) */
    double ring_radius;     /* R [m]; the ring must lie inside the grid */
    int32_t nx, ny;         /* grid size (3..4096 each) */
    double h;               /* pixel pitch [m] */
    int32_t n_rays;         /* rays per fan (2..4096), take-off angles
                               th = phi_t + pi - pi/2 + (i + 1/2) pi / n_rays */
    double ds;              /* RK4 arclength step [m] */
    int32_t max_steps;      /* step cap per ray; a ray still inside is "lost" */
    double support_margin;  /* the update is zero outside |x| <= R - support_margin */
    double c_ref;           /* reference (water) speed [m/s] for traveltime residuals */
    double f_ref;           /* frequency [Hz] at which c is the phase speed */
    double power_y;         /* absorption power law alpha = alpha0 f_MHz^y */
} rb_geometry;

/* Last vertex of one ray, where it crosses the ring (device records). */
typedef struct rb_ray_end {
    double t;               /* traveltime [s] */
    double t_res;           /* t - |x_end - x_t| / c_ref */
    double x, y;            /* crossing point [m] */
    float theta;            /* direction [rad] */
    float q;                /* ray-tube width per radian of take-off angle (J = |q|) */
    float p;                /* dynamic ray-tracing partner of q */
    float l;                /* integral of alpha0 along the ray */
    int32_t kappa;          /* KMAH index: sign changes of q after the first step */
    int32_t n_vert;         /* vertices including this one; -1 if the ray was lost */
} rb_ray_end;               /* 56 bytes */

/* Ray output of rb_trace_rays.  ends is required ([n_elem][n_rays]); the
 * per-vertex arrays are optional (all NULL or all set), each
 * [n_elem][n_rays][max_steps + 1]; entries past a ray's n_vert are unset. */
typedef struct rb_rays {
    rb_ray_end* ends;
    float* vx;              /* vertex position */
    float* vy;
    double* vt;             /* traveltime */
    float* vq;
    float* vl;
    int32_t* vkappa;
} rb_rays;

/* One gridded entry, table[t][pixel] (16 bytes, 16-byte aligned).  tkey is
 * the order-preserving bit pattern of the float T_res (traveltime minus
 * |p - x_t| / c_ref): for tkey >= 0x80000000 the float bits are
 * tkey & 0x7fffffff, otherwise ~tkey.  tag = (triangle id << 8) | min(kappa, 255),
 * triangle id = (i * (max_steps + 1) + k) * 2 + half.  q is the interpolated
 * tube width (J = max(|q|, h/4)), l the interpolated alpha0 integral.  A hole
 * (no ray triangle covers the pixel, or the pixel is outside the support)
 * has tkey = tag = 0xffffffff. */
typedef struct rb_cell {
    uint32_t tag;
    uint32_t tkey;
    float q;
    float l;
} rb_cell;

/* Stages of one update, in launch order (for optional stage timing). */
typedef enum {
    RB_STAGE_FIELDS = 0,    /* derivative grids */
    RB_STAGE_TRACE_GRID,    /* fused ray fans + first-arrival gridding */
    RB_STAGE_LINK,          /* ray linking, residuals, data weights */
    RB_STAGE_IMAGES,        /* tensor-core operand images of the set (BF16X3; empty for FP32) */
    RB_STAGE_ADJOINT,       /* Born adjoint + Hessian diagonal over the set */
    RB_STAGE_DIRECTION,     /* eps, direction, numerator of the step */
    RB_STAGE_FORWARD,       /* Born forward of the direction over the set (step mode exact) */
    RB_STAGE_APPLY,         /* step, c update, norm */
    RB_STAGE_COUNT
} rb_stage;

typedef struct rb_update_params {
    double outlier_frac;    /* fraction of kept data zeroed by largest |residual| (0.01) */
    double eps_rel;         /* eps = eps_rel * mean over the support of sum_w H_w (1e-3) */
    int32_t step_mode;      /* rb_step_mode */
    int32_t tune;           /* kernel-shape choices, 0 = the library's rules (a caller may time the
                               alternatives and pass the fastest; the results do not change):
                               bits 0-1 the rasteriser's work mapping, 1 = warps along the ray tubes,
                               2 = warps across them (rule: along from tubes of 4 pixels at the ring);
                               bits 2-3 the tensor-core adjoint, 1 = CTA pairs (cta_group::2 MMAs),
                               2 = one CTA per pixel tile (the rule); other bits 0; a field of 3
                               returns RB_ERR_ARG */
    void* stage_events;     /* NULL, or a caller-created array of 2 * RB_STAGE_COUNT cudaEvent_t:
                               events [2s] and [2s+1] are recorded on the stream before and after
                               stage s (no events are created or destroyed by the library) */
} rb_update_params;

/* Device-side diagnostics of one update (written by rb_hf_update). */
typedef struct rb_diag {
    double dc_norm;         /* ||dc||_2 over the support */
    double alpha;           /* step scale (1 for RB_STEP_DIAG) */
    double eps;             /* the eps used in the solution-space weight */
    uint32_t lost_rays;
    uint32_t holes;         /* support pixels no triangle covered, summed over fans */
    uint32_t unlinked;      /* masked (e, r) pairs no ray interval bracketed */
    uint32_t kept;          /* masked, linked data entries over the set */
    uint32_t zeroed;        /* of those, zeroed as outliers */
    uint32_t tc_timeouts;   /* tensor-core pipeline waits that ran out (0 unless the device misbehaves) */
} rb_diag;                  /* 48 bytes */

/* Largest n_freq per call to rb_green_grid / rb_ray_forward / rb_hf_update / rb_cg_update. */
#define RB_MAX_FREQ 16
/* Largest number of CG iterations per call to rb_cg_update (the paper cites 10-15). */
#define RB_MAX_CG 24

/*
 * Bytes of workspace every call below needs for this geometry, n_freq
 * frequencies and precision (one size fits all entry points).  Returns 0 for
 * an invalid geometry.  The workspace must be 256-byte aligned.
 */
size_t rb_workspace_size(const rb_geometry* geom, int32_t n_freq, rb_precision prec);

/*
 * Ray fans (Eqs. 6-7 via their characteristics and dynamic ray tracing): for
 * every element t, n_rays rays integrated by RK4 in arclength from x_t through
 * the sound speed c[ny*nx] (with absorption alpha0[ny*nx] integrated along the
 * ray) until they cross the ring.  Fills out->ends and, if set, the vertex arrays.
 */
rb_status rb_trace_rays(const rb_geometry* geom, const float* c, const float* alpha0, rb_rays* out,
                        void* ws, size_t ws_bytes, rb_stream stream);

/*
 * Green's-function gridding ("back-propagation of ray parameters", Sec. 5):
 * traces the fans again and rasterises every ray-tube triangle onto the
 * support pixels, keeping per (t, pixel) the first arrival, into
 * tables[n_elem][ny*nx].  If g_out is not NULL, also writes the Green's
 * functions of Eqs. 4-5, g_out[n_freq][n_elem][ny*nx] complex, for the host
 * array freqs_hz[n_freq] (n_freq in 1..RB_MAX_FREQ; ignored when g_out is NULL).
 */
rb_status rb_green_grid(const rb_geometry* geom, const float* c, const float* alpha0, rb_cell* tables,
                        const double* freqs_hz, int32_t n_freq, float* g_out,
                        void* ws, size_t ws_bytes, rb_stream stream);

/*
 * Ray-model data at the receivers (the p(c) of Eq. 8, by ray linking): for
 * each emitter e and receiver r the ray interval of fan e whose end angles
 * bracket r (first arrival if several), interpolated, and the Green's
 * function evaluated there.  ends from rb_trace_rays; freqs_hz is a host
 * array; p_out[n_freq][n_elem][n_elem] complex (zero when unlinked);
 * linked_out[n_elem][n_elem] (nullable) is 1 where a bracket was found.
 */
rb_status rb_ray_forward(const rb_geometry* geom, const float* c, const rb_ray_end* ends,
                         const double* freqs_hz, int32_t n_freq, float* p_out, uint8_t* linked_out,
                         rb_stream stream);

/*
 * Residuals and data-space weights of one frequency set (Eq. 8 and Sec. 4.1),
 * the data side of rb_hf_update on its own: rays through c[ny*nx], ray-model
 * data by ray linking, R = p_ray - p_obs, and the weights W: 1 for receivers
 * on the opposite ~75 % of the ring (circular index distance >= ceil(n_elem/8))
 * that a ray interval links, then the floor(outlier_frac * kept) kept entries
 * of largest |R| over the whole set zeroed (ties to the smallest flat index
 * (w, e, r)).  p_obs, resid_out [n_freq][n_elem][n_elem] complex;
 * w_out [n_freq][n_elem][n_elem] bytes (0 or 1); freqs_hz host array, n_freq
 * in 1..RB_MAX_FREQ; outlier_frac in [0, 1).  Workspace as
 * rb_workspace_size(geom, n_freq, RB_PREC_FP32).
 */
rb_status rb_data_weights(const rb_geometry* geom, const float* c, const float* alpha0, const double* freqs_hz,
                          int32_t n_freq, const float* p_obs, double outlier_frac, float* resid_out, uint8_t* w_out,
                          void* ws, size_t ws_bytes, rb_stream stream);

/*
 * Born forward operator (the linearisation of Eq. 10 in Born form):
 *   d[e][r] = w^2 sum_x G_e(x) G_r(x) m(x),  w = 2 pi f_hz,
 * with G from tables and c (Eqs. 4-5); m[ny*nx] real; d_out[n_elem][n_elem] complex.
 */
rb_status rb_born_forward(const rb_geometry* geom, const rb_cell* tables, const float* c, double f_hz,
                          const float* m, float* d_out, rb_precision prec,
                          void* ws, size_t ws_bytes, rb_stream stream);

/*
 * Born adjoint (gradient of Eq. 8) and Gauss-Newton Hessian diagonal:
 *   g(x) = w^2 sum_{e,r} conj(G_e(x) G_r(x)) W[e][r] R[e][r]     -> g_out[ny*nx] complex
 *   H(x) = w^4 sum_{e,r} W[e][r] |G_e(x)|^2 |G_r(x)|^2            -> hdiag_out[ny*nx] (nullable)
 * resid[n_elem][n_elem] complex, w[n_elem][n_elem] bytes (0 or 1).
 */
rb_status rb_born_adjoint(const rb_geometry* geom, const rb_cell* tables, const float* c, double f_hz,
                          const float* resid, const uint8_t* w, float* g_out, float* hdiag_out,
                          rb_precision prec, void* ws, size_t ws_bytes, rb_stream stream);

/*
 * One Hessian-free ray-Born update over one set of consecutive frequencies
 * (Secs. 3-4): rays and tables in c, ray-model data and residuals
 * R = p_ray - p_obs, data weights (opposite-75 % receiver mask, linked pairs,
 * largest outlier_frac of |R| zeroed), the diagonal-Hessian direction
 * -sum_w Re g_w / (sum_w H_w + eps) on the support, its step scale, then
 * c_inout += dc.  p_obs[n_freq][n_elem][n_elem] complex; freqs_hz host array;
 * dc_out[ny*nx] (nullable); diag_out device record (nullable).
 */
rb_status rb_hf_update(const rb_geometry* geom, float* c_inout, const float* alpha0, const double* freqs_hz,
                       int32_t n_freq, const float* p_obs, const rb_update_params* params, rb_precision prec,
                       float* dc_out, rb_diag* diag_out, void* ws, size_t ws_bytes, rb_stream stream);

/*
 * CG variant of the frequency-set update (Sec. 3: the linear equation of Eq. 10
 * solved iteratively by conjugate gradients, 10-15 iterations per set, as in
 * the earlier ray-Born method the one-step update replaces).  Everything up to
 * the gradient is as in rb_hf_update (same rays, data weights and eps); then
 * cg_iters iterations (1..RB_MAX_CG) of preconditioned conjugate gradients on
 *   A dm = -sum_w Re g_w,   A = sum_w Re(B_w^H W B_w)   (support pixels, dm_0 = 0),
 * each one Born forward per frequency and one adjoint over the set, with the
 * operand images of the set built once and reused.  precond 1: M^-1 = 1/(sum_w
 * H_w + eps) per pixel (one iteration then equals rb_hf_update's exact step);
 * precond 0: plain CG (run with the scalar 1/(mean H + eps), which leaves the
 * iterates unchanged).  Then dc = -dm c^3 / (2 h^2), c_inout += dc.
 * params->step_mode must be valid and is otherwise ignored.  cg_hist_out
 * (nullable, device, cg_iters + 1 doubles) receives rho_k / rho_0 with
 * rho_k = <r_k, M^-1 r_k>.  diag_out as for rb_hf_update (alpha = 1).  Stage
 * events: RB_STAGE_DIRECTION brackets the CG start, RB_STAGE_FORWARD all
 * iterations.  Same workspace size as rb_hf_update.  Errors as rb_hf_update,
 * plus RB_ERR_ARG for cg_iters or precond out of range.
 */
rb_status rb_cg_update(const rb_geometry* geom, float* c_inout, const float* alpha0, const double* freqs_hz,
                       int32_t n_freq, const float* p_obs, const rb_update_params* params, int32_t cg_iters,
                       int32_t precond, rb_precision prec, float* dc_out, double* cg_hist_out, rb_diag* diag_out,
                       void* ws, size_t ws_bytes, rb_stream stream);

/*
 * Times of flight along rays (Sec. 4, the measured quantity of the time-of-flight
 * initial guess): the first-arrival traveltime of the ray linking of every pair,
 * as in rb_ray_forward, through c[ny*nx].  t_out[n_elem][n_elem] double (device,
 * 0 where unlinked); linked_out[n_elem][n_elem] (nullable) 1 where linked.
 */
rb_status rb_tof_times(const rb_geometry* geom, const float* c, const float* alpha0, double* t_out,
                       uint8_t* linked_out, void* ws, size_t ws_bytes, rb_stream stream);

/* Largest n_iter of rb_tof_invert. */
#define RB_MAX_TOF_ITERS 16

/*
 * Time-of-flight initial guess (Sec. 4: a few linearisations of a reconstruction
 * that fits measured times of flight with times along rays; the paper uses three).
 * Each linearisation traces the fans through c_inout, links them, and takes one
 * SIRT step in slowness along the rays (ds = D_col^-1 L^T D_row^-1 (t_obs - T(c))
 * with L the ray-path operator of the linked times; rows: the opposite ~75 % of
 * the ring, linked in the data (obs_linked) and in c); c_inout <- 1/(1/c + ds) on
 * the support.  t_obs, obs_linked [n_elem][n_elem] device (e.g. from
 * rb_tof_times).  resid_out (nullable, device, n_iter + 1 doubles): RMS ToF
 * misfit of the rows before each linearisation and after the last.  n_iter in
 * 1..RB_MAX_TOF_ITERS.  Workspace as rb_workspace_size(geom, 1, RB_PREC_FP32).
 */
rb_status rb_tof_invert(const rb_geometry* geom, float* c_inout, const float* alpha0, const double* t_obs,
                        const uint8_t* obs_linked, int32_t n_iter, double* resid_out, void* ws, size_t ws_bytes,
                        rb_stream stream);

/*
 * Born forward operator without a workspace (the paper has no counterpart:
 * this is a calling convention of the library).  For callers that cannot
 * give the library device scratch memory, such as plugins of a host
 * framework that passes in its own tensors but no allocator, or real-time
 * loops that forbid device allocation once running.  Computes the same
 * d[e][r] = w^2 sum_x G_e(x) G_r(x) m(x) as rb_born_forward (FP32), from
 * tables, c and m into d_out[n_elem][n_elem] complex, and allocates nothing.
 *
 * Its scratch is one fixed device array of RB_NOALLOC_SCRATCH_BYTES inside
 * the library, held on every device that loads the library until the process
 * exits.  The first call on each device looks up the array's device address
 * (make that first call before any stream capture).  All calls share the
 * array: calls whose kernels overlap on the GPU race and must be serialised
 * by the caller.  Sizes whose scratch does not fit (n_elem^2 * 8 bytes above
 * RB_NOALLOC_SCRATCH_BYTES - 16 KiB) return RB_ERR_SHAPE; with the current
 * size every n_elem <= 1024 fits.  Errors are returned as for rb_born_forward.
 */
#define RB_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u + 16u * 1024u)
rb_status rb_born_forward_noalloc(const rb_geometry* geom, const rb_cell* tables, const float* c, double f_hz,
                                  const float* m, float* d_out, rb_stream stream);

/* Static description of a status code. */
const char* rb_status_string(rb_status s);

#ifdef __cplusplus
}
#endif

#endif /* RB_H */
