// noalloc.cu -- a residual entry point that allocates no device memory.
//
// Every other entry point of this library works on a plan, and creating a
// plan calls cudaMalloc for its workspace.  Some callers cannot do that: a
// serving process that forbids device allocation after start-up (an
// allocation can synchronise the device and take unbounded time in the
// middle of a latency budget), or code running under a framework whose
// caching allocator already holds all of the GPU's memory.  For them,
// eecmg_residual_noalloc computes r = g - H u and its norms with the same
// convolution kernel as a level solve's first step, and keeps its scratch
// (the PSF taps, the per-block partial sums of the deterministic reduction
// and the reduction's scalars) in one file-scope __device__ array of fixed
// size, which every GPU that loads the library holds until the process
// exits.  The caller passes only inputs and outputs.
#include <mutex>
#include <string>

#include "launch.hpp"
#include "plan.hpp"

namespace eecmg {
namespace {

// Largest image side accepted (both sides); bounds the partial-sum count.
constexpr int NOALLOC_MAX_SIDE = 4096;
constexpr unsigned int NOALLOC_MAX_BLOCKS =
    ((NOALLOC_MAX_SIDE + CONV_TW - 1) / CONV_TW) * ((NOALLOC_MAX_SIDE + CONV_TH - 1) / CONV_TH);

struct NoallocScratch {
    Scalars sc;
    Taps taps;
    double partials[NOALLOC_MAX_BLOCKS * NPART];
};

// The scratch: about 264 KB per device, shared by every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Device address of the scratch array, looked up once per device (host code
// may not use the symbol itself: in host code it names a host-side stand-in).
std::mutex g_mu;
void* g_scratch_addr[128] = {};

eecmg_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_residual_noalloc: cudaGetDevice: ") +
                                             cudaGetErrorString(e));
    if (dev < 0 || dev >= 128)
        return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_residual_noalloc: device ordinal >= 128");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(EECMG_ERR_CUDA,
                             std::string("eecmg_residual_noalloc: cudaGetSymbolAddress: ") +
                                 cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return EECMG_OK;
}

// Installs this call's taps and clears the reduction state (the counter of
// the last-block reduction must start at zero).
__global__ void k_noalloc_setup(Taps t, NoallocScratch* s) {
    const int n = (int)(sizeof(Taps) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(&t);
    int* dst = reinterpret_cast<int*>(&s->taps);
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        Scalars z{};
        s->sc = z;
    }
}

__global__ void k_noalloc_norms(const NoallocScratch* s, double* out) {
    out[0] = s->sc.rr;
    out[1] = s->sc.gg;
}

}  // namespace
}  // namespace eecmg

using namespace eecmg;

extern "C" eecmg_status eecmg_residual_noalloc(int width, int height, const double* psf,
                                               int psf_w, int psf_h, const float* g,
                                               const float* u, float* r, double* norms,
                                               cudaStream_t stream) {
    if (width < 1 || height < 1 || width > NOALLOC_MAX_SIDE || height > NOALLOC_MAX_SIDE)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_residual_noalloc: width and height must be in [1, 4096]");
    if (!psf || psf_w < 1 || psf_h < 1 || !(psf_w & 1) || !(psf_h & 1) ||
        psf_w / 2 > EECMG_MAX_RADIUS || psf_h / 2 > EECMG_MAX_RADIUS)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_residual_noalloc: PSF must be non-NULL, odd-sized, radius <= 12");
    if (!g || !u || !r || !norms || r == g || r == u)
        return set_error(EECMG_ERR_INVALID_ARG,
                         "eecmg_residual_noalloc: NULL or aliased buffers");
    void* base = nullptr;
    eecmg_status st = scratch_address(&base);
    if (st != EECMG_OK) return st;
    NoallocScratch* s = static_cast<NoallocScratch*>(base);

    // correlation-form taps of H: C(dy, dx) = K(-dy, -dx), non-zero entries only
    Taps t{};
    const int ry = psf_h / 2, rx = psf_w / 2;
    t.ry = ry;
    t.rx = rx;
    t.rt = ry > rx ? ry : rx;
    t.sep = 0;
    int n = 0;
    for (int dy = -ry; dy <= ry; ++dy)
        for (int dx = -rx; dx <= rx; ++dx) {
            const double v = psf[(size_t)(-dy + ry) * psf_w + (-dx + rx)];
            if (v != 0.0) {
                t.dy[n] = dy;
                t.dx[n] = dx;
                t.wt[n] = (float)v;
                ++n;
            }
        }
    t.ntap = n;

    k_noalloc_setup<<<1, 256, 0, stream>>>(t, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_residual_noalloc: ") + cudaGetErrorString(e));
    ConvArgs a;
    a.x = u;
    a.y = r;
    a.e0 = g;
    a.taps = &s->taps;
    a.sc = &s->sc;
    a.partials = s->partials;
    a.h = height;
    a.w = width;
    a.mode = CM_RESID;
    e = launch_conv(a, t.rt, 0, 0, stream);
    if (e != cudaSuccess)
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_residual_noalloc: ") + cudaGetErrorString(e));
    k_noalloc_norms<<<1, 1, 0, stream>>>(s, norms);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(EECMG_ERR_CUDA, std::string("eecmg_residual_noalloc: ") + cudaGetErrorString(e));
    return EECMG_OK;
}
