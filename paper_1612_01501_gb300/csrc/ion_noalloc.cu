// ion_noalloc.cu -- dense gap-junction currents without any device allocation.
//
// ion_gj_dense needs one scratch buffer per call: a copy of V_dend padded to a multiple
// of 256 floats (the padding holds a sentinel voltage so padded pairs contribute zero),
// which it takes from the stream-ordered allocator.  Some callers must not allocate:
// a loop that has to finish every 50 us step on time (allocation can block and
// synchronise), code running while a stream is being captured into a CUDA graph, and
// host programs whose device memory is owned by their own allocator.  For them this
// file keeps the scratch in a fixed device array instead.
//
// The array lives for as long as the library is loaded, on every GPU that loads it
// (NOALLOC_MAX_CELLS floats = 256 KiB per device).  Host code cannot pass the array's
// name to a kernel (on the host that name is only a stand-in, not a device address), so
// the first call on each device looks up its device address with cudaGetSymbolAddress,
// with that device current, and caches it together with the identity of the device's
// context.  A device reset destroys the context and the module with it; the next call
// sees a different context and looks the address up again (that call, like the first,
// should come before any stream capture).
#include <cuda_runtime.h>

#include <mutex>

#include "ion.h"
#include "ion_kernels.cuh"
#include "ion_sim.h"

namespace {

constexpr int NOALLOC_MAX_CELLS = 65536;   // padded V_dend capacity (multiple of 256)
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) float g_noalloc_vdend[NOALLOC_MAX_CELLS];

// Driver entry points that identify the current context (resolved through the runtime,
// so the library needs no link-time dependence on the driver library).  Both return a
// CUresult (0 = success); a context is an opaque pointer.
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);

struct Slot {
    float *ptr = nullptr;            // device address of this device's array
    unsigned long long ctx_id = 0;   // the context it belongs to (0: unknown)
};

std::mutex g_noalloc_mu;
Slot g_slot[MAX_DEVICES];
bool g_resolved = false;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Unique id of the calling thread's current context, or 0 where the driver cannot tell.
unsigned long long current_ctx_id() {
    if (!g_resolved) {
        g_resolved = true;
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current == nullptr || g_ctx_id == nullptr || g_ctx_current(&ctx) != 0 || ctx == nullptr ||
        g_ctx_id(ctx, &id) != 0)
        return 0;
    return id;
}

// Device address of this device's copy of the array: looked up once per device and
// context (again after a reset gave the device a new context).
cudaError_t noalloc_scratch(int dev, float **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    Slot &sl = g_slot[dev];
    const unsigned long long id = current_ctx_id();
    if (sl.ptr == nullptr || (id != 0 && id != sl.ctx_id)) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_vdend);
        if (e != cudaSuccess) return e;
        sl.ptr = static_cast<float *>(p);
        sl.ctx_id = id;
    }
    *out = sl.ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" ion_status ion_gj_dense_noalloc(const float *vdend, int32_t n, float g_c, float *ic, int32_t kahan,
                                           void *stream) {
    if (!vdend || !ic || n < 1) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_gj_dense_noalloc: bad arguments");
    const int n_pad = (n + ion::PAD_J - 1) / ion::PAD_J * ion::PAD_J;
    if (n_pad > NOALLOC_MAX_CELLS)
        return ion_fail(nullptr, ION_ERR_INVALID_ARG,
                        "ion_gj_dense_noalloc: n = %d needs %d scratch floats, the fixed array holds %d "
                        "(use ion_gj_dense for larger networks)",
                        n, n_pad, NOALLOC_MAX_CELLS);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_gj_dense_noalloc: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES)
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_gj_dense_noalloc: device ordinal %d too large", dev);
    float *pad = nullptr;
    e = noalloc_scratch(dev, &pad);
    if (e != cudaSuccess)
        return ion_fail(nullptr, ION_ERR_CUDA, "ion_gj_dense_noalloc: scratch lookup: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    // every call rewrites the whole padded range it uses: V_dend, then the sentinel tail
    e = cudaMemcpyAsync(pad, vdend, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = ion::launch_fill(pad + n, ion::PAD_VOLT, n_pad - n, st);
    int R, W, GJ;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ion_choose_dense_shape(n, sms, &R, &W, &GJ);
    if (e == cudaSuccess) e = ion::prepare_dense_step(R, W, GJ, n_pad);
    if (e == cudaSuccess) {
        ion::DenseArgs a{};
        a.c.n = n;
        a.c.n_pad = n_pad;
        a.g = g_c;
        a.kahan = kahan ? 1 : 0;
        a.fuse = 0;
        a.ic_out = ic;
        a.vd_in = pad;
        e = ion::launch_dense_step(a, R, W, GJ, st);
    }
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_gj_dense_noalloc: %s", cudaGetErrorString(e));
    return ION_OK;
}
