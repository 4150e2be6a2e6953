// hf_noalloc.cu -- hf_fields_noalloc: energy and force for one rotation with
// no device allocation at all.
//
// Who needs this: callers that are not allowed to allocate device memory
// once they are running.  A haptic servo loop has about 1 ms per frame, and
// cudaMalloc / cudaFree may synchronise the device and take far longer than
// that.  A plug-in living inside a host application whose memory manager owns
// all device memory may only use the buffers it is handed.  A runtime that
// forbids dynamic allocation after start-up is in the same position.  Such a
// caller owns the two density grids and the four output fields; everything
// the pipeline needs between them lives in one file-scope device array.
//
// Properties of that array:
//   * size: 4 half-spectrum buffers of the largest supported grid
//     (N <= HF_NOALLOC_MAX_N = 64: 4 x 64*64*33 complex64 = 4.3 MB) plus the
//     two rotation matrices; every GPU that loads the library holds it until
//     the process exits;
//   * it is shared by every call: calls whose GPU work overlaps (different
//     streams, or host threads) race on it and give wrong results, so keep
//     them ordered on one stream or serialise them;
//   * each call overwrites every element it later reads, so nothing has to
//     be cleared between calls even though the array keeps the previous
//     call's contents.
// The first call on a device is the set-up, and it is not allocation-free:
// with CUDA's default lazy module loading, the device code of this file (the
// array included) and of the pass kernels is loaded onto the device only
// when first used, so the first call loads those modules -- reserving the
// array -- when it looks up the array's device address
// (cudaGetSymbolAddress) with that device current, and it sets the kernels'
// shared-memory limits.  Make one warm-up call per device at start-up,
// before the time-critical loop and before any stream capture; the calls
// after it allocate nothing.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "hf.h"
#include "hf_internal.h"

namespace {

constexpr int kMaxN = HF_NOALLOC_MAX_N;
constexpr size_t kMaxHalfSpec = (size_t)kMaxN * kMaxN * (kMaxN / 2 + 1);  // complex elements
constexpr size_t kRotOffset = 4 * kMaxHalfSpec * sizeof(float2);         // bytes
constexpr size_t kScratchBytes = kRotOffset + 256;
constexpr int kMaxDevices = 64;

// The only scratch of hf_fields_noalloc.  In host code this name is a
// host-side stand-in, not a device address: host code must use the address
// from cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// failures are reported through hf_last_error(), like every other entry point
hf_status noalloc_fail(hf_status s, const char *fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    hf::set_last_error(msg);
    return s;
}

// Device address of the scratch array on the current device; the first call
// per device resolves it and sets the pass kernels' shared-memory limits.
hf_status scratch_on_current_device(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(HF_ECUDA, "hf_fields_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HF_EUNSUPPORTED, "hf_fields_noalloc: device %d", dev);
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(HF_ECUDA, "hf_fields_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        for (int n = 32; n <= kMaxN; n *= 2) {
            e = hf::fft_init_attrs(n);
            if (e != cudaSuccess)
                return noalloc_fail(HF_ECUDA, "hf_fields_noalloc: kernel set-up: %s", cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return HF_OK;
}

// the identity and the call's rotation, written by the GPU from kernel
// arguments (no host buffer has to outlive the call)
__global__ void write_rotations(hf::Rot9 a, hf::Rot9 b, float *dst) {
    const int i = threadIdx.x;
    if (i < 9) {
        dst[i] = a.r[i];
        dst[9 + i] = b.r[i];
    }
}

}  // namespace

extern "C" hf_status hf_fields_noalloc(int n, const float *d_rho1, const float *d_rho2, const float h_quat[4],
                                       float *d_E, float *d_Fx, float *d_Fy, float *d_Fz, hf_stream stream) {
    if (n != 32 && n != 64)
        return noalloc_fail(HF_EINVAL, "hf_fields_noalloc: N=%d is not supported; the static scratch holds grids "
                                       "of N=32 or N=64 (maximum N=%d)", n, kMaxN);
    if (!d_rho1 || !d_rho2 || !h_quat || !d_E || !d_Fx || !d_Fy || !d_Fz)
        return noalloc_fail(HF_EINVAL, "hf_fields_noalloc: NULL argument");
    double w = h_quat[0], x = h_quat[1], y = h_quat[2], z = h_quat[3];
    const double nq = sqrt(w * w + x * x + y * y + z * z);
    if (!(nq > 0.0) || !isfinite(nq)) return noalloc_fail(HF_EINVAL, "hf_fields_noalloc: quaternion is zero or not finite");
    w /= nq; x /= nq; y /= nq; z /= nq;
    const double M[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                         2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
    hf::Rot9 ident = {{1, 0, 0, 0, 1, 0, 0, 0, 1}}, rot;
    for (int k = 0; k < 9; ++k) rot.r[k] = (float)M[k];

    void *base = nullptr;
    hf_status s = scratch_on_current_device(&base);
    if (s != HF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t he = hf::half_spec_elems(n);
    float2 *spec = (float2 *)base, *X1 = spec + he, *Y1 = X1 + he, *Y2 = Y1 + he;
    float *rot9 = (float *)((unsigned char *)base + kRotOffset);  // [identity | rotation]
    // (h^3 / N^3) in float64, rounded once, as for a stationary part
    const double h = 2.0 / n;
    const float scale = (float)(h * h * h / ((double)n * n * n));
    hf::FieldPtrs out{d_E, d_Fx, d_Fy, d_Fz, 0};

    cudaError_t e;
    (void)cudaGetLastError();  // drop a stale non-sticky error before checking the launches
    write_rotations<<<1, 32, 0, st>>>(ident, rot, rot9);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = hf::run_passA(n, d_rho1, rot9, X1, 1, st)) != cudaSuccess ||
        (e = hf::run_passB_forward(n, X1, spec, scale, st)) != cudaSuccess ||
        (e = hf::run_passA(n, d_rho2, rot9 + 9, X1, 1, st)) != cudaSuccess ||
        (e = hf::run_passB(n, X1, spec, Y1, Y2, 1, st)) != cudaSuccess ||
        (e = hf::run_passC(n, Y1, Y2, out, 1, st)) != cudaSuccess)
        return noalloc_fail(HF_ECUDA, "hf_fields_noalloc: launch failed: %s", cudaGetErrorString(e));
    return HF_OK;
}
