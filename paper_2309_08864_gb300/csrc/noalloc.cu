// noalloc.cu -- so2dr_run_device_noalloc: the in-core stencil run for callers
// that may not allocate memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they want a stencil sweep: code running while a CUDA graph is being
// captured, real-time loops that forbid allocation after start-up, and
// host runtimes that only hand out pre-registered device buffers.  This entry
// point takes the caller's device input and output and keeps its one scratch
// grid (the ping-pong partner of the output) in a file-scope device array.
#include <cuda_runtime.h>

#include <atomic>
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
std::mutex g_setup_mutex;                        // guards the one-time set-up below
std::atomic<void*> g_scratch_addr[kMaxDevices];  // device address of the array, per device

// In host code the array's name is only a host-side stand-in; the address a
// kernel may use comes from cudaGetSymbolAddress with the device current.
int scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(SO2DR_E_UNSUPPORTED, "device index above 63");
    void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
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
    if (plane > (int64_t)kScratchBytes / esize || n0 > (int64_t)kScratchBytes / esize / plane)
        return set_error(SO2DR_E_INFEASIBLE,
                         "grid larger than the 32 MiB scratch of so2dr_run_device_noalloc");
    if (steps == 0 || n0 <= 2 * radius) {
        cudaError_t e = cudaMemcpyAsync(d_out, d_in, (size_t)(n0 * plane * esize), cudaMemcpyDeviceToDevice,
                                        static_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? SO2DR_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    void* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;

    const int shape = kind == SO2DR_BOX ? kBox2D : (ndim == 3 ? kStar3D : kStar2D);
    const int csize = dtype == SO2DR_F64 ? 8 : 4;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    // launch depths as in Algorithm 1 (k_on-step launches, then the residual);
    // the last launch writes d_out, the ones before alternate with scratch
    const int64_t nfull = steps / k_on, res = steps % k_on, L = nfull + (res ? 1 : 0);
    const void* src = d_in;
    for (int64_t j = 0; j < L; ++j) {
        const int depth = (j < nfull) ? k_on : (int)res;
        void* dst = ((L - 1 - j) % 2 == 0) ? d_out : scratch;
        LaunchShape ls = stencil_launch_shape(shape, radius, depth, ny, nx, csize, (int)esize);
        if (!ls.ok) return set_error(SO2DR_E_UNSUPPORTED, "fused depth too large for the stencil kernel");
        ls.grid.z = 1;
        if (ls.fast) {
            int occ = stencil_occupancy(dtype, shape, radius, depth, ls);
            ls.grid.z = (unsigned)choose_segments((int64_t)ls.grid.x * ls.grid.y, n0, radius, depth, sms, occ);
        }
        StencilArgs a;
        std::memset(&a, 0, sizeof(a));
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
