// Host-side internals shared by the libmgq translation units: argument
// checks, error reporting, workspace layout, precision dispatch and the
// deterministic FP64 reductions.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "mgq.h"
#include "mgq_device.cuh"

namespace mgq {

// ---- tracing: an NVTX range for the lifetime of the object (a no-op unless a
// profiler is attached)
struct Trace {
    explicit Trace(const char* name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;
};

// ---- errors
mgq_status fail(mgq_status s, const char* fmt, ...);
mgq_status cuda_check(const char* where);  // cudaGetLastError after launches

// ---- geometry / sizes
bool valid_dims(const int32_t dims[4]);
Geom make_geom(const int32_t dims[4]);
uint64_t site_stride(const int32_t dims[4]);
int planes_of(int prec);  // complex planes per link: 9 or 6
uint64_t links_bytes(const mgq_lattice* lat);
uint64_t alg_bytes(const mgq_lattice* lat);

// Workspace layout: [partials | scalars | link copy | algebra field]
constexpr size_t WS_PARTIALS = 0;
constexpr size_t WS_NPARTIALS = 8192;  // doubles
constexpr size_t WS_SCALARS = WS_NPARTIALS * sizeof(double);
constexpr size_t WS_NSCALARS = 512;  // doubles
constexpr size_t WS_LINKS = WS_SCALARS + WS_NSCALARS * sizeof(double);
inline uint64_t round256(uint64_t b) { return (b + 255) & ~uint64_t(255); }
uint64_t ws_alg_offset(const mgq_lattice* lat);
uint64_t workspace_bytes(const mgq_lattice* lat);
inline double* ws_partials(const mgq_lattice* lat) { return reinterpret_cast<double*>((char*)lat->work + WS_PARTIALS); }
inline double* ws_scalars(const mgq_lattice* lat) { return reinterpret_cast<double*>((char*)lat->work + WS_SCALARS); }
inline void* ws_links(const mgq_lattice* lat) { return (char*)lat->work + WS_LINKS; }
inline void* ws_alg(const mgq_lattice* lat) { return (char*)lat->work + ws_alg_offset(lat); }

// Validates a lattice descriptor; need_work additionally checks the workspace.
mgq_status check_lattice(const mgq_lattice* lat, bool need_work, const char* fn);

// Copies n device doubles to a host or device destination; a host
// destination synchronises the stream.
mgq_status deliver(const double* dev_src, double* out, size_t n, cudaStream_t st, const char* fn);
mgq_status deliver_int(const int* dev_src, int* out, size_t n, cudaStream_t st, const char* fn);
bool is_device_ptr(const void* p);

// Number of blocks used by the site-parallel reduction kernels.
int reduction_blocks(int V, int threads);
// threads per block of a tunable kernel (mgq_kernel) for a precision
constexpr int MGQ_NKERNELS = 5;
int block_size(int kernel, int prec);

// Sums n partials in a fixed order into out[0] * scale (device).
void launch_final_sum(const double* partials, int n, double scale, double* out, cudaStream_t st);

// launchers shared between translation units
mgq_status plaquette_into(const mgq_lattice* lat, double* partials, double* dev_out, cudaStream_t st);
mgq_status heatbath_subsweep(mgq_lattice* lat, double beta, uint64_t sweep, int n_hb, int mu, int par, uint8_t* dec,
                             cudaStream_t st);
mgq_status overrelax_subsweep(mgq_lattice* lat, int mu, int par, cudaStream_t st);
// E (site average) and Q of the clover field strength into dev_out[0], dev_out[1]
mgq_status clover_into(const mgq_lattice* lat, double* partials, double* dev_out, cudaStream_t st);
// Per-block E and Q partial sums (E at partials[0..nb), Q at partials[nb..2nb));
// skipped when gate != nullptr and *gate == 0.  Returns nb.
int clover_partials(const mgq_lattice* lat, double* partials, const int* gate, cudaStream_t st);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// launch with programmatic stream serialisation (see pdl_wait)
template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, (KArgs)args...);
}

// launch with programmatic stream serialisation and dynamic shared memory
template <class... KArgs, class... Args>
inline void launch_pdl_smem(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, (KArgs)args...);
}


template <class T, int NP>
inline Links<T, NP> links_of(const mgq_lattice* lat) {
    Links<T, NP> l;
    l.p = reinterpret_cast<Cx<T>*>(lat->links);
    l.S = (int)site_stride(lat->dims);
    return l;
}
template <class T, int NP>
inline Links<T, NP> links_at(void* p, const int32_t dims[4]) {
    Links<T, NP> l;
    l.p = reinterpret_cast<Cx<T>*>(p);
    l.S = (int)site_stride(dims);
    return l;
}
template <class T>
inline Alg<T> alg_at(void* p, const int32_t dims[4]) {
    Alg<T> a;
    a.p = reinterpret_cast<T*>(p);
    a.S = (int)site_stride(dims);
    return a;
}

// Calls F.template operator()<T, NP>() for the lattice's precision.
template <class F>
inline void dispatch_prec(int prec, F&& f) {
    switch (prec) {
        case MGQ_F64: f.template operator()<double, 9>(); break;
        case MGQ_F32: f.template operator()<float, 9>(); break;
        default: f.template operator()<float, 6>(); break;
    }
}

// Calls f.template operator()<MU>() for a run-time direction mu.
template <class F>
inline void dispatch_mu(int mu, F&& f) {
    switch (mu) {
        case 0: f.template operator()<0>(); break;
        case 1: f.template operator()<1>(); break;
        case 2: f.template operator()<2>(); break;
        default: f.template operator()<3>(); break;
    }
}

// Block-wide FP64 sum in a fixed order (warp shuffles then shared memory);
// the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_part[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? warp_part[threadIdx.x] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

}  // namespace mgq
