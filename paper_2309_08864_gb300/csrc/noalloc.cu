// noalloc.cu -- so2dr_run_device_noalloc: the in-core stencil run for callers
// that may not allocate memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they want a stencil sweep: code running while a CUDA graph is being
// captured, real-time loops that forbid allocation after start-up, and
// host runtimes that only hand out pre-registered device buffers.  This entry
// point takes the caller's device input and output and keeps its one scratch
// grid (the ping-pong partner of the output) in a file-scope device array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "kernels.hpp"
#include "plan.hpp"
#include "run.hpp"

using namespace so2dr;

namespace {

// Scratch of the allocation-free entry point.  Every GPU that loads the
// library holds these bytes until the process exits.
constexpr size_t kScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// Device address of the array per device, with the context it was looked up
// in: a reset of the device (cudaDeviceReset) or any re-creation of its
// primary context reloads the module, and the array may then sit elsewhere.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    void* ptr = nullptr;
};
std::mutex g_scratch_mutex;
ScratchAddr g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 when it cannot be
// read: the address is then looked up again on every call).
unsigned long long current_context_id() {
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        else
            cudaGetLastError();
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        else
            cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// In host code the array's name is only a host-side stand-in; the address a
// kernel may use comes from cudaGetSymbolAddress with the device current.
int scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(SO2DR_E_UNSUPPORTED, "device index above 63");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchAddr& s = g_scratch[dev];
    if (!s.ptr || ctx == 0 || s.ctx_id != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        s.ptr = p;
        s.ctx_id = ctx;
    }
    *out = s.ptr;
    return SO2DR_OK;
}

}  // namespace

extern "C" int so2dr_run_device_noalloc(int ndim, const int64_t* dims, int radius, int kind,
                                        const double* coeffs, int ncoeffs, int64_t steps, int k_on,
                                        int dtype, const void* d_in, void* d_out, void* stream) {
    // ---- argument checks (no CUDA call, no allocation)
    if (ndim != 2 && ndim != 3) return set_error(SO2DR_E_INVAL, "ndim must be 2 or 3");
    if (!dims || !coeffs || !d_in || !d_out) return set_error(SO2DR_E_INVAL, "NULL argument");
    if (d_in == d_out) return set_error(SO2DR_E_INVAL, "d_in and d_out must be different buffers");
    if (reinterpret_cast<uintptr_t>(d_in) % 16 || reinterpret_cast<uintptr_t>(d_out) % 16)
        return set_error(SO2DR_E_INVAL, "d_in and d_out must be 16-byte aligned");
    if (radius < 1 || radius > kMaxRadius) return set_error(SO2DR_E_INVAL, "radius must be 1..4");
    if (kind != SO2DR_STAR && !(kind == SO2DR_BOX && ndim == 2))
        return set_error(SO2DR_E_UNSUPPORTED, "constant-coefficient star (2D/3D) or 2D box stencils only");
    const int64_t esize = elem_size(dtype);
    if (esize == 0) return set_error(SO2DR_E_INVAL, "unknown storage dtype");
    if (steps < 0) return set_error(SO2DR_E_INVAL, "steps must be >= 0");
    if (k_on < 1 || k_on > kMaxKon) return set_error(SO2DR_E_INVAL, "k_on must be 1..16");
    const int nc = num_coeffs(ndim, radius, kind);
    if (ncoeffs != nc) return set_error(SO2DR_E_INVAL, "coefficient count does not match the stencil");
    int64_t n0 = dims[0], ny = ndim == 3 ? dims[1] : 1, nx = ndim == 3 ? dims[2] : dims[1];
    if (n0 < 1 || ny < 1 || nx < 1) return set_error(SO2DR_E_INVAL, "dims must be >= 1");
    if (n0 > ((int64_t)1 << 31) || ny > ((int64_t)1 << 31) || nx > ((int64_t)1 << 31))
        return set_error(SO2DR_E_UNSUPPORTED, "axis too long");
    const int64_t plane = ny * nx;
    if (plane > ((int64_t)1 << 40) / esize || n0 > ((int64_t)1 << 40) / esize / plane)
        return set_error(SO2DR_E_UNSUPPORTED, "grid too large");
    const uintptr_t bytes = (uintptr_t)(n0 * plane * esize);
    const uintptr_t pi = reinterpret_cast<uintptr_t>(d_in), po = reinterpret_cast<uintptr_t>(d_out);
    if (pi < po + bytes && po < pi + bytes) return set_error(SO2DR_E_INVAL, "d_in and d_out overlap");
    if (steps == 0 || n0 <= 2 * radius) {
        cudaError_t e = cudaMemcpyAsync(d_out, d_in, (size_t)bytes, cudaMemcpyDeviceToDevice,
                                        static_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? SO2DR_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    // launch depths: floor(steps / k_on) launches of depth k_on, then one of
    // the remainder; the last launch writes d_out and the ones before it
    // alternate between d_out and the scratch array, so a single launch needs
    // no scratch at all
    const int64_t nfull = steps / k_on, res = steps % k_on, L = nfull + (res ? 1 : 0);
    void* scratch = nullptr;
    if (L >= 2) {
        if ((int64_t)bytes > (int64_t)kScratchBytes)
            return set_error(SO2DR_E_INFEASIBLE,
                             "grid larger than the 32 MiB scratch of so2dr_run_device_noalloc "
                             "(runs of more than one launch only)");
        int rc = scratch_for_current_device(&scratch);
        if (rc) return rc;
    }

    const int shape = kind == SO2DR_BOX ? kBox2D : (ndim == 3 ? kStar3D : kStar2D);
    const int csize = dtype == SO2DR_F64 ? 8 : 4;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    const void* src = d_in;
    for (int64_t j = 0; j < L; ++j) {
        const int depth = (j < nfull) ? k_on : (int)res;
        void* dst = ((L - 1 - j) % 2 == 0) ? d_out : scratch;
        LaunchShape ls = stencil_launch_shape(shape, radius, depth, ny, nx, csize, (int)esize);
        if (!ls.ok) return set_error(SO2DR_E_UNSUPPORTED, "fused depth too large for the stencil kernel");
        ls.grid.z = 1;
        StencilArgs a;
        std::memset(&a, 0, sizeof(a));
        if (ls.fast) {
            int occ = stencil_occupancy(dtype, shape, radius, depth, ls);
            if (ls.fast == kFastStar3D) choose_work_split(ls, n0, radius, depth, sms, occ, &a.split);
            else ls.grid.z = (unsigned)choose_segments((int64_t)ls.grid.x * ls.grid.y, n0, radius, depth, sms, occ, false);
        }
        a.in = src;
        a.in_cap = n0;
        a.in_slot0 = 0;
        a.in_lo = 0;
        a.in_hi = n0;
        a.out = dst;
        a.out_lo = 0;
        a.out_hi = n0;
        a.n0 = n0;
        a.ny = ny;
        a.nx = nx;
        a.depth = depth;
        a.edge_lo = a.edge_hi = 1;
        a.lx = ls.lx;
        a.ly = ls.ly;
        a.tx = ls.tx;
        a.ty = ls.ty;
        for (int k = 0; k < nc && k < kMaxCoeffsDev; ++k) {
            a.c[k] = coeffs[k];
            a.cf[k] = (float)coeffs[k];
            a.cf2[k] = make_float2(a.cf[k], a.cf[k]);
        }
        cudaError_t e = launch_stencil(dtype, shape, radius, a, ls, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(e, "stencil launch");
        src = dst;
    }
    return SO2DR_OK;
}
