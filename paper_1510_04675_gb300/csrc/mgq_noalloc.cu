// mgq_plaquette_noalloc: the average plaquette for callers that cannot give
// the library any device memory.
//
// mgq_plaquette reduces its per-block partial sums in the caller's workspace.
// Some callers cannot provide one: code that runs under another framework's
// memory manager which already owns the device memory and forbids further
// cudaMalloc calls, or a latency-critical monitoring hook where cudaMalloc /
// cudaFree would implicitly synchronise the device.  This entry point keeps
// its scratch in a fixed array of this library instead, so it needs only the
// links and the output.
//
// The scratch array below is static device memory: every GPU that loads
// libmgq holds its 64 KiB until the process exits.
#include <mutex>

#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// One partial sum per block of 256 sites, plus one slot for the result.
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_PARTIALS = 8191;
constexpr long NOALLOC_MAX_SITES = (long)NOALLOC_MAX_PARTIALS * NOALLOC_THREADS;  // 2,096,896 sites

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_PARTIALS + 1];

// Device address of g_noalloc_scratch per device.  Outside stream capture it
// is looked up on every call (so a context re-created after cudaDeviceReset is
// picked up); under capture the address of the last call outside capture on
// that device is used, because the lookup may load the module, which capture
// forbids.
constexpr int NOALLOC_MAX_DEVICES = 64;
static double* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_scratch_mutex;

static mgq_status scratch_for_current_device(cudaStream_t st, double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_check("mgq_plaquette_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(MGQ_EUNSUPPORTED, "mgq_plaquette_noalloc: device %d beyond %d", dev, NOALLOC_MAX_DEVICES);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return cuda_check("mgq_plaquette_noalloc: cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cap != cudaStreamCaptureStatusNone && !g_scratch_addr[dev])
        return fail(MGQ_EINVAL, "mgq_plaquette_noalloc: the first call on a device must come before any stream capture");
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(MGQ_ECUDA, "mgq_plaquette_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return MGQ_OK;
}

// One block per NOALLOC_THREADS sites (no grid stride), so the partial count
// is ceil(V / NOALLOC_THREADS) and every slot the final sum reads is written
// by this launch: nothing in the shared scratch needs clearing.
template <class T, int NP>
__global__ void __launch_bounds__(NOALLOC_THREADS) k_plaquette_noalloc(Links<T, NP> U, Geom g, double* partials) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (idx < g.V) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        acc = site_plaquettes(U, g, par, h);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_plaquette_noalloc(const mgq_lattice* lat, double* plaq_out, void* stream) {
    // the workspace is not used, so it is not checked
    mgq_status s = check_lattice(lat, false, "mgq_plaquette_noalloc");
    if (s) return s;
    if (!plaq_out) return fail(MGQ_EINVAL, "mgq_plaquette_noalloc: plaq_out is NULL");
    const Geom g = make_geom(lat->dims);
    if ((long)g.V > NOALLOC_MAX_SITES)
        return fail(MGQ_EINVAL,
                    "mgq_plaquette_noalloc: %d sites exceed the %ld-site limit of its fixed scratch "
                    "(use mgq_plaquette with a workspace)",
                    g.V, NOALLOC_MAX_SITES);
    cudaStream_t st = as_stream(stream);
    double* scratch = nullptr;
    if ((s = scratch_for_current_device(st, &scratch))) return s;
    const int nb = (g.V + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_plaquette_noalloc<T, NP><<<nb, NOALLOC_THREADS, 0, st>>>(links_of<T, NP>(lat), g, scratch);
    });
    launch_final_sum(scratch, nb, 1.0 / (18.0 * (double)g.V), scratch + NOALLOC_MAX_PARTIALS, st);
    if ((s = cuda_check("mgq_plaquette_noalloc"))) return s;
    return deliver(scratch + NOALLOC_MAX_PARTIALS, plaq_out, 1, st, "mgq_plaquette_noalloc");
}

}  // extern "C"
