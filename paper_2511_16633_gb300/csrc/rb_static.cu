// rb_born_forward_noalloc: the Born forward operator without any workspace.
//
// Some callers of this library cannot hand it device scratch memory: plugins
// of a host framework that passes in its own input and output tensors but no
// allocator, or real-time loops that forbid any device allocation once they
// are running.  For them this entry point keeps its scratch (the element
// positions and the split-K partial sums of the contraction) in one
// file-scope device array of fixed size, reserved when the library's module
// is loaded on a device and held until the process exits.
//
// The array's name is only a host-side stand-in in host code; kernels get
// its device address, looked up once per device with cudaGetSymbolAddress
// while that device is current.  The lookup happens in the first call on
// each device (so that call should come before any stream capture).
// Every call shares the array: calls whose kernels overlap on the GPU (two
// streams, or two host threads on one device) race on it and must be
// serialised by the caller.  Nothing in the array needs to start at zero:
// each call writes every entry it later reads.
#include <mutex>

#include "rb_internal.cuh"

namespace {

constexpr size_t kElemBytes = 16u * 1024u;                    // [n_elem <= 1024] float4 positions
constexpr size_t kPartialBytes = (size_t)RB_NOALLOC_SCRATCH_BYTES - kElemBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[RB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool geom_ok_noalloc(const rb_geometry* g) {
    // the same geometry rules as the workspace entry points, via the layout query
    WsLayout L;
    return rb_ws_layout(g, 1, RB_PREC_FP32, &L) != 0;
}

}  // namespace

extern "C" rb_status rb_born_forward_noalloc(const rb_geometry* geom, const rb_cell* tables, const float* c,
                                             double f_hz, const float* m, float* d_out, rb_stream stream) {
    if (!geom || !tables || !c || !m || !d_out) return RB_ERR_ARG;
    if (!(f_hz > 0.0) || !isfinite(f_hz)) return RB_ERR_ARG;
    if (!geom_ok_noalloc(geom)) return RB_ERR_SHAPE;
    const size_t ne2 = (size_t)geom->n_elem * geom->n_elem;
    const size_t per_chunk = ne2 * sizeof(float2);
    if ((size_t)geom->n_elem * 16 > kElemBytes || per_chunk > kPartialBytes) return RB_ERR_SHAPE;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return RB_ERR_CUDA;
    float4* exy = (float4*)base;
    float2* partial = (float2*)((char*)base + kElemBytes);
    int nch = rb_fwd_chunks_for(geom->nx * geom->ny);
    const int fit = (int)(kPartialBytes / per_chunk);
    if (nch > fit) nch = fit;
    const GeoDev G = rb_make_geo(geom, exy);
    const FreqC F = rb_make_freq(geom, f_hz);
    cudaStream_t s = (cudaStream_t)stream;
    if (launch_elem_positions(G, exy, s) != cudaSuccess) return RB_ERR_CUDA;
    if (launch_forward_simt(G, tables, c, F, m, partial, nch, s) != cudaSuccess) return RB_ERR_CUDA;
    if (launch_forward_reduce(G, F, partial, nch, (float2*)d_out, nullptr, nullptr, s) != cudaSuccess)
        return RB_ERR_CUDA;
    return RB_OK;
}
