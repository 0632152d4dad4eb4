// libmgq core: errors, sizes, field initialisation and layout conversion,
// the checkerboard heat-bath and overrelaxation sub-sweeps (Sec. IV.A),
// the plaquette (Sec. III) and the unitarity check.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// =============================================================== host utilities
static thread_local char g_err[512] = "";

mgq_status fail(mgq_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

mgq_status cuda_check(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MGQ_ECUDA, "%s: %s", where, cudaGetErrorString(e));
    return MGQ_OK;
}

bool valid_dims(const int32_t dims[4]) {
    if (!dims) return false;
    uint64_t V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (dims[mu] < 2 || (dims[mu] & 1)) return false;
        V *= (uint64_t)dims[mu];
    }
    // every index a kernel forms in 32 bits (links 4V, algebra entries 8 V/2,
    // plaquettes 6V / 2) stays below 2^31
    return V <= (uint64_t(1) << 28);
}

uint64_t site_stride(const int32_t dims[4]) {
    if (!valid_dims(dims)) return 0;
    uint64_t Vh = (uint64_t)dims[0] * dims[1] * dims[2] * dims[3] / 2;
    return (Vh + 63) & ~uint64_t(63);
}

Geom make_geom(const int32_t dims[4]) {
    Geom g;
    for (int mu = 0; mu < 4; mu++) g.L[mu] = dims[mu];
    g.V = dims[0] * dims[1] * dims[2] * dims[3];
    g.Vh = g.V / 2;
    g.S = (int)site_stride(dims);
    set_divisors(g);
    return g;
}

int planes_of(int prec) { return prec == MGQ_F32_C12 ? 6 : 9; }

static int real_bytes(int prec) { return prec == MGQ_F64 ? 8 : 4; }

uint64_t links_bytes(const mgq_lattice* lat) {
    if (!lat || !valid_dims(lat->dims) || lat->prec < 0 || lat->prec > 2) return 0;
    return 4ull * 2ull * planes_of(lat->prec) * site_stride(lat->dims) * 2ull * real_bytes(lat->prec);
}

uint64_t alg_bytes(const mgq_lattice* lat) {
    if (!lat || !valid_dims(lat->dims) || lat->prec < 0 || lat->prec > 2) return 0;
    return 4ull * 2ull * 8ull * site_stride(lat->dims) * real_bytes(lat->prec);
}

uint64_t ws_alg_offset(const mgq_lattice* lat) { return WS_LINKS + round256(links_bytes(lat)); }

uint64_t workspace_bytes(const mgq_lattice* lat) {
    uint64_t lb = links_bytes(lat);
    if (!lb) return 0;
    return ws_alg_offset(lat) + round256(alg_bytes(lat));
}

mgq_status check_lattice(const mgq_lattice* lat, bool need_work, const char* fn) {
    if (!lat) return fail(MGQ_EINVAL, "%s: lattice is NULL", fn);
    if (!valid_dims(lat->dims))
        return fail(MGQ_EINVAL, "%s: extents %d x %d x %d x %d must be even, >= 2, volume <= 2^28", fn, lat->dims[0],
                    lat->dims[1], lat->dims[2], lat->dims[3]);
    for (int mu = 0; mu < 4; mu++) {
        if (lat->bc[mu] == MGQ_OPEN) return fail(MGQ_EUNSUPPORTED, "%s: only periodic boundary conditions are built", fn);
        if (lat->bc[mu] != MGQ_PERIODIC) return fail(MGQ_EINVAL, "%s: bc[%d] = %d is not an mgq_bc", fn, mu, lat->bc[mu]);
    }
    if (lat->prec < MGQ_F64 || lat->prec > MGQ_F32_C12) return fail(MGQ_EINVAL, "%s: prec %d invalid", fn, lat->prec);
    if (lat->action != MGQ_WILSON) return fail(MGQ_EUNSUPPORTED, "%s: only the Wilson action is built", fn);
    if (lat->reserved != 0) return fail(MGQ_EINVAL, "%s: reserved field must be 0", fn);
    if (!lat->links) return fail(MGQ_EINVAL, "%s: links is NULL", fn);
    if (((uintptr_t)lat->links & 15) != 0) return fail(MGQ_EINVAL, "%s: links must be 16-byte aligned", fn);
    if (need_work) {
        if (!lat->work) return fail(MGQ_EINVAL, "%s: workspace is NULL", fn);
        if (((uintptr_t)lat->work & 255) != 0) return fail(MGQ_EINVAL, "%s: workspace must be 256-byte aligned", fn);
        if (lat->work_bytes < workspace_bytes(lat))
            return fail(MGQ_ENOMEM, "%s: workspace has %llu bytes, needs %llu", fn, (unsigned long long)lat->work_bytes,
                        (unsigned long long)workspace_bytes(lat));
    }
    return MGQ_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class V>
static mgq_status deliver_t(const V* src, V* out, size_t n, cudaStream_t st, const char* fn) {
    if (!out || n == 0) return MGQ_OK;
    if (is_device_ptr(out)) {
        if (cudaMemcpyAsync(out, src, n * sizeof(V), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return cuda_check(fn);
        return MGQ_OK;
    }
    if (cudaMemcpyAsync(out, src, n * sizeof(V), cudaMemcpyDeviceToHost, st) != cudaSuccess) return cuda_check(fn);
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(fn);
    return MGQ_OK;
}

mgq_status deliver(const double* src, double* out, size_t n, cudaStream_t st, const char* fn) {
    return deliver_t(src, out, n, st, fn);
}
mgq_status deliver_int(const int* src, int* out, size_t n, cudaStream_t st, const char* fn) {
    return deliver_t(src, out, n, st, fn);
}

int reduction_blocks(int V, int threads) {
    int b = (V + threads - 1) / threads;
    return b < 1184 ? b : 1184;  // 152 SMs x 8
}

// =============================================================== reductions
__global__ void k_final_sum(const double* __restrict__ partials, int n, double scale, double* out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
    v = block_sum(v);
    if (threadIdx.x == 0) out[0] = v * scale;
}

void launch_final_sum(const double* partials, int n, double scale, double* out, cudaStream_t st) {
    k_final_sum<<<1, 512, 0, st>>>(partials, n, scale, out);
}

// =============================================================== fields
template <class T, int NP>
__global__ void k_init(Links<T, NP> U, Geom g, int start, RngKey rk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * g.V) return;
    const int mu = idx / g.V, rem = idx - mu * g.V, par = rem >= g.Vh, h = rem - par * g.Vh;
    M3<T> u;
    if (!start) {
        u = unit3<T>();
    } else {
        int x[4];
        cb_coords(g, par, h, x);
        const uint32_t lex = (uint32_t)lex_of(g, x);
        // 18 unit normals (Box-Muller on pairs of uniforms), Gram-Schmidt
        T gs[20];
#pragma unroll
        for (int call = 0; call < 5; call++) {
            uint4 r = draw(rk, lex, (uint32_t)mu, 0u, (uint32_t)call, KIND_HOT);
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int p = 0; p < 2; p++) {
                T u0 = u01<T>(w[2 * p]), u1 = u01<T>(w[2 * p + 1]);
                T rad = m_sqrt(T(-2) * m_log(u0));
                T sn, cs;
                m_sincospi(T(2) * u1, &sn, &cs);
                gs[4 * call + 2 * p] = rad * cs;
                gs[4 * call + 2 * p + 1] = rad * sn;
            }
        }
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) u.e[r][c] = mk(gs[2 * (3 * r + c)], gs[2 * (3 * r + c) + 1]);
        reunitarize(u);
    }
    U.store(mu, par, h, u);
}

// canonical double[V][4][3][3][2] <-> lattice layout
template <class T, int NP>
__global__ void k_import(Links<T, NP> U, Geom g, const double* __restrict__ canon) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * g.V) return;
    const int lex = idx >> 2, mu = idx & 3;
    int x[4];
    int r = lex;
    for (int m = 0; m < 4; m++) { x[m] = r % g.L[m]; r /= g.L[m]; }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double* src = canon + (size_t)idx * 18;
    M3<T> u;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) u.e[a][b] = mk((T)src[(a * 3 + b) * 2], (T)src[(a * 3 + b) * 2 + 1]);
    U.store(mu, par, lex >> 1, u);
}

template <class T, int NP>
__global__ void k_export(Links<T, NP> U, Geom g, double* __restrict__ canon) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * g.V) return;
    const int lex = idx >> 2, mu = idx & 3;
    int x[4];
    int r = lex;
    for (int m = 0; m < 4; m++) { x[m] = r % g.L[m]; r /= g.L[m]; }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    M3<T> u = U.load(mu, par, lex >> 1);
    double* dst = canon + (size_t)idx * 18;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            dst[(a * 3 + b) * 2] = (double)u.e[a][b].re;
            dst[(a * 3 + b) * 2 + 1] = (double)u.e[a][b].im;
        }
}

// One thread per link of the (MU, par) subset; MU is a template parameter so
// that every neighbour index is resolved at compile time.  Four resident
// blocks of 128 threads per SM (at most 128 registers) measured fastest.
// FAST: the instance for one heat-bath attempt per subgroup without decision
// recording (the benchmarked setting); the compiler removes the attempt loop
// and the recording code.
template <class T, int NP, int MU, bool FAST>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 4) k_heatbath(Links<T, NP> U, Geom g, int par, T beta, RngKey rk, int n_hb,
                                                    uint8_t* __restrict__ dec) {
    if constexpr (FAST) {
        n_hb = 1;
        dec = nullptr;
    }
    pdl_launch_dependents();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h >= g.Vh) return;
    const M3<T> A = staple(U, g, x, h, MU, par);
    M3<T> u = U.load(MU, par, h);
    const int lex = lex_of(g, x);
    hb_link(u, A, beta, n_hb, rk, (uint32_t)lex, (uint32_t)MU, dec ? dec + ((size_t)lex * 4 + MU) * 3 : nullptr);
    U.store(MU, par, h, u);
}

template <class T, int NP, int MU>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 4) k_overrelax(Links<T, NP> U, Geom g, int par) {
    pdl_launch_dependents();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h >= g.Vh) return;
    const M3<T> A = staple(U, g, x, h, MU, par);
    M3<T> u = U.load(MU, par, h);
    or_link(u, A);
    U.store(MU, par, h, u);
}

// FP32 12-real instances with the staple's links staged through shared memory
// (staple_staged): the loads of each half-term are in flight during the
// previous one's arithmetic; STAGED_THREADS threads per block (the tuned block
// size does not apply), STAGED_SMEM bytes of dynamic shared memory.
template <int MU>
__global__ void __launch_bounds__(STAGED_THREADS, 5) k_heatbath_staged(Links<float, 6> U, Geom g, int par, float beta, RngKey rk) {
    extern __shared__ float4 sm[];
    pdl_launch_dependents();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h >= g.Vh) return;
    M3<float> u;
    uint4 r[3];
    const uint32_t lex = (uint32_t)lex_of(g, x);
    // the three Philox draws while the first staged loads are in flight
    const M3<float> A = staple_staged(U, g, x, h, MU, par, sm, u, [&]() {
#pragma unroll
        for (int s = 0; s < 3; s++) r[s] = draw(rk, lex, (uint32_t)MU, (uint32_t)s, 0u, KIND_HB);
    });
    hb_link_drawn(u, A, beta, r);
    U.store(MU, par, h, u);
}

template <int MU>
__global__ void __launch_bounds__(STAGED_THREADS, 5) k_overrelax_staged(Links<float, 6> U, Geom g, int par) {
    extern __shared__ float4 sm[];
    pdl_launch_dependents();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h >= g.Vh) return;
    M3<float> u;
    const M3<float> A = staple_staged(U, g, x, h, MU, par, sm, u);
    or_link(u, A);
    U.store(MU, par, h, u);
}

__global__ void __launch_bounds__(STAGED_THREADS, 4)
    k_overrelax_last_staged(Links<float, 6> U, Geom g, int par, double* __restrict__ partials) {
    extern __shared__ float4 sm[];
    pdl_launch_dependents();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h < g.Vh) {
        M3<float> u;
        const M3<float> A = staple_staged(U, g, x, h, 3, par, sm, u);
        if (par == 1) acc = (double)retr_nn(u, A);
        or_link(u, A);
        U.store(3, par, h, u);
        acc += site_plaquettes<float, 6, 3>(U, g, par, h);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}


// The two sub-sweeps of direction 3, which end an overrelaxation sweep, with
// the plaquette of the field they leave folded in (per-block FP64 partials).
// Neither sub-sweep writes directions 0-2, so each adds the plaquettes of the
// planes of directions 0, 1, 2 at the sites of its parity.  Every plaquette of
// a plane (3, nu) holds exactly one direction-3 link of odd parity, and the
// six plaquettes through U_3(x) sum to Re Tr(U_3(x) A_3(x)), which
// overrelaxation leaves unchanged: the parity-1 sub-sweep adds it, taken
// before the update, for each of its links.
template <class T, int NP>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : 4)
    k_overrelax_last(Links<T, NP> U, Geom g, int par, double* __restrict__ partials) {
    pdl_launch_dependents();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h < g.Vh) {
        const M3<T> A = staple(U, g, x, h, 3, par);
        M3<T> u = U.load(3, par, h);
        if (par == 1) acc = (double)retr_nn(u, A);
        or_link(u, A);
        U.store(3, par, h, u);
        acc += site_plaquettes<T, NP, 3>(U, g, par, h);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// =============================================================== plaquette
template <class T, int NP>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_plaquette(Links<T, NP> U, Geom g, double* __restrict__ partials) {
    double acc = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        acc += site_plaquettes(U, g, par, h);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// =============================================================== unitarity
template <class T, int NP>
__global__ void k_unitarity(Links<T, NP> U, Geom g, double* __restrict__ partials) {
    double m = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 4 * g.V; idx += gridDim.x * blockDim.x) {
        const int mu = idx / g.V, rem = idx - mu * g.V, par = rem >= g.Vh, h = rem - par * g.Vh;
        M3<T> u = U.load(mu, par, h);
        M3<T> uu = mul_nd(u, u);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double dr = (double)uu.e[i][j].re - (i == j ? 1.0 : 0.0), di = (double)uu.e[i][j].im;
                m = fmax(m, fmax(fabs(dr), fabs(di)));
            }
        // det = row0 . (row1 x row2)
        Cx<T> c0 = u.e[1][1] * u.e[2][2] - u.e[1][2] * u.e[2][1];
        Cx<T> c1 = u.e[1][2] * u.e[2][0] - u.e[1][0] * u.e[2][2];
        Cx<T> c2 = u.e[1][0] * u.e[2][1] - u.e[1][1] * u.e[2][0];
        Cx<T> det = u.e[0][0] * c0 + u.e[0][1] * c1 + u.e[0][2] * c2;
        m = fmax(m, hypot((double)det.re - 1.0, (double)det.im));
    }
    __shared__ double sm[256];
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

__global__ void k_final_max(const double* __restrict__ partials, int n, double* out) {
    __shared__ double sm[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, partials[i]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

// =============================================================== launchers
static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// Launch shape of the sub-sweep kernels per (kernel, precision): threads per
// block, at most the 128 the kernels are compiled for.  Set by
// mgq_set_block_size (the autotuner); 128 by default.
static int g_block[MGQ_NKERNELS][3] = {{128, 128, 128}, {128, 128, 128}, {128, 128, 128}, {128, 128, 128},
                                      {128, 128, 128}};

int block_size(int kernel, int prec) { return g_block[kernel][prec]; }

mgq_status heatbath_subsweep(mgq_lattice* lat, double beta, uint64_t sweep, int n_hb, int mu, int par,
                             uint8_t* dec, cudaStream_t st) {
    Trace trace("heatbath_subsweep");
    const Geom g = make_geom(lat->dims);
    const int bs = g_block[MGQ_KERNEL_HEATBATH][lat->prec];
    const RngKey rk = make_rng(lat->seed, lat->lattice_id, sweep);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        dispatch_mu(mu, [&]<int MU>() {
            if constexpr (sizeof(T) == 4 && NP == 6) {
                if (n_hb == 1 && !dec && g.Vh >= STAGED_MIN_VH) {
                    launch_pdl_smem(k_heatbath_staged<MU>, nblk(g.Vh, STAGED_THREADS), STAGED_THREADS, STAGED_SMEM, st,
                                    links_of<T, NP>(lat), g, par, (float)beta, rk);
                    return;
                }
            }
            if (n_hb == 1 && !dec)
                launch_pdl(k_heatbath<T, NP, MU, true>, nblk(g.Vh, bs), bs, st, links_of<T, NP>(lat), g, par,
                           (T)beta, rk, n_hb, dec);
            else
                launch_pdl(k_heatbath<T, NP, MU, false>, nblk(g.Vh, bs), bs, st, links_of<T, NP>(lat), g, par,
                           (T)beta, rk, n_hb, dec);
        });
    });
    return cuda_check("mgq_heatbath");
}

mgq_status overrelax_subsweep(mgq_lattice* lat, int mu, int par, cudaStream_t st) {
    Trace trace("overrelax_subsweep");
    const Geom g = make_geom(lat->dims);
    const int bs = g_block[MGQ_KERNEL_OVERRELAX][lat->prec];
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        dispatch_mu(mu, [&]<int MU>() {
            if (sizeof(T) == 4 && NP == 6 && g.Vh >= STAGED_MIN_VH)
                launch_pdl_smem(k_overrelax_staged<MU>, nblk(g.Vh, STAGED_THREADS), STAGED_THREADS, STAGED_SMEM, st,
                                links_of<float, 6>(lat), g, par);
            else
                launch_pdl(k_overrelax<T, NP, MU>, nblk(g.Vh, bs), bs, st, links_of<T, NP>(lat), g, par);
        });
    });
    return cuda_check("mgq_overrelax");
}

// One overrelaxation sweep whose last two sub-sweeps also measure the
// plaquette of the result into dev_out[0] (device); needs the workspace.
mgq_status overrelax_sweep_plaquette(mgq_lattice* lat, double* dev_out, cudaStream_t st) {
    mgq_status s;
    for (int mu = 0; mu < 3; mu++)
        for (int par = 0; par < 2; par++)
            if ((s = overrelax_subsweep(lat, mu, par, st))) return s;
    Trace trace("overrelax_last");
    const Geom g = make_geom(lat->dims);
    const bool staged = lat->prec == MGQ_F32_C12 && g.Vh >= STAGED_MIN_VH;
    const int bs = staged ? STAGED_THREADS : g_block[MGQ_KERNEL_OVERRELAX][lat->prec];
    const int nb = nblk(g.Vh, bs);
    double* partials = reinterpret_cast<double*>(ws_alg(lat));  // free during sweeps; >= 2 nb doubles
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        for (int par = 0; par < 2; par++) {
            if (staged)
                launch_pdl_smem(k_overrelax_last_staged, nb, STAGED_THREADS, STAGED_SMEM, st,
                                links_of<float, 6>(lat), g, par, partials + par * nb);
            else
                launch_pdl(k_overrelax_last<T, NP>, nb, bs, st, links_of<T, NP>(lat), g, par, partials + par * nb);
        }
    });
    launch_final_sum(partials, 2 * nb, 1.0 / (18.0 * (double)g.V), dev_out, st);
    return cuda_check("overrelax_sweep_plaquette");
}

// plaquette of `links` into dev_out[0] (device)
mgq_status plaquette_into(const mgq_lattice* lat, double* partials, double* dev_out, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    const int nb = reduction_blocks(g.V, 256);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_plaquette<T, NP><<<nb, 256, 0, st>>>(links_of<T, NP>(lat), g, partials);
    });
    launch_final_sum(partials, nb, 1.0 / (18.0 * (double)g.V), dev_out, st);
    return cuda_check("mgq_plaquette");
}

}  // namespace mgq

using namespace mgq;

// =============================================================== C ABI
extern "C" {

int mgq_abi_version(void) { return MGQ_ABI_VERSION; }

const char* mgq_status_string(mgq_status s) {
    switch (s) {
        case MGQ_OK: return "ok";
        case MGQ_EINVAL: return "invalid argument";
        case MGQ_ENOMEM: return "workspace too small";
        case MGQ_ECUDA: return "CUDA error";
        case MGQ_EUNSUPPORTED: return "unsupported";
        case MGQ_ETIMEOUT: return "device wait timed out";
        case MGQ_ENONUNITARY: return "non-unitary link";
    }
    return "unknown status";
}

const char* mgq_last_error(void) { return g_err; }

uint64_t mgq_site_stride(const int32_t dims[4]) { return site_stride(dims); }
uint64_t mgq_links_bytes(const mgq_lattice* lat) { return links_bytes(lat); }
uint64_t mgq_mom_bytes(const mgq_lattice* lat) { return alg_bytes(lat); }
uint64_t mgq_workspace_bytes(const mgq_lattice* lat) { return workspace_bytes(lat); }

mgq_status mgq_set_block_size(int kernel, int prec, int threads) {
    if (kernel < 0 || kernel >= MGQ_NKERNELS) return fail(MGQ_EINVAL, "mgq_set_block_size: unknown kernel %d", kernel);
    if (prec < MGQ_F64 || prec > MGQ_F32_C12) return fail(MGQ_EINVAL, "mgq_set_block_size: prec %d invalid", prec);
    if (threads < 32 || threads > 128 || (threads & 31))
        return fail(MGQ_EINVAL, "mgq_set_block_size: threads must be 32, 64, 96 or 128");
    g_block[kernel][prec] = threads;
    return MGQ_OK;
}

int mgq_get_block_size(int kernel, int prec) {
    if (kernel < 0 || kernel >= MGQ_NKERNELS || prec < MGQ_F64 || prec > MGQ_F32_C12) return 0;
    return g_block[kernel][prec];
}

mgq_status mgq_init_links(mgq_lattice* lat, int start, void* stream) {
    Trace trace("mgq_init_links");
    mgq_status s = check_lattice(lat, false, "mgq_init_links");
    if (s) return s;
    if (start != 0 && start != 1) return fail(MGQ_EINVAL, "mgq_init_links: start must be 0 (cold) or 1 (hot)");
    const Geom g = make_geom(lat->dims);
    const RngKey rk = make_rng(lat->seed, lat->lattice_id, 0);
    cudaStream_t st = as_stream(stream);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_init<T, NP><<<nblk(4L * g.V, 128), 128, 0, st>>>(links_of<T, NP>(lat), g, start, rk);
    });
    return cuda_check("mgq_init_links");
}

mgq_status mgq_import_links(mgq_lattice* lat, const double* canon, void* stream) {
    mgq_status s = check_lattice(lat, false, "mgq_import_links");
    if (s) return s;
    if (!canon || !is_device_ptr(canon)) return fail(MGQ_EINVAL, "mgq_import_links: canon must be a device pointer");
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_import<T, NP><<<nblk(4L * g.V, 128), 128, 0, st>>>(links_of<T, NP>(lat), g, canon);
    });
    return cuda_check("mgq_import_links");
}

mgq_status mgq_export_links(const mgq_lattice* lat, double* canon, void* stream) {
    mgq_status s = check_lattice(lat, false, "mgq_export_links");
    if (s) return s;
    if (!canon || !is_device_ptr(canon)) return fail(MGQ_EINVAL, "mgq_export_links: canon must be a device pointer");
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_export<T, NP><<<nblk(4L * g.V, 128), 128, 0, st>>>(links_of<T, NP>(lat), g, canon);
    });
    return cuda_check("mgq_export_links");
}

static mgq_status check_hb_args(double beta, int n_hb, const char* fn) {
    if (!(beta > 0.0) || beta > 1e6) return fail(MGQ_EINVAL, "%s: beta must be in (0, 1e6]", fn);
    if (n_hb < 1 || n_hb > 256) return fail(MGQ_EINVAL, "%s: n_hb must be in [1, 256]", fn);
    return MGQ_OK;
}

mgq_status mgq_heatbath_subsweep(mgq_lattice* lat, double beta, uint64_t sweep, int n_hb, int mu, int parity,
                                 uint8_t* decisions, void* stream) {
    mgq_status s = check_lattice(lat, false, "mgq_heatbath_subsweep");
    if (s) return s;
    if ((s = check_hb_args(beta, n_hb, "mgq_heatbath_subsweep"))) return s;
    if (mu < 0 || mu > 3 || parity < 0 || parity > 1) return fail(MGQ_EINVAL, "mgq_heatbath_subsweep: bad mu/parity");
    return heatbath_subsweep(lat, beta, sweep, n_hb, mu, parity, decisions, as_stream(stream));
}

mgq_status mgq_heatbath_sweep(mgq_lattice* lat, double beta, uint64_t sweep, int n_hb, void* stream) {
    Trace trace("mgq_heatbath_sweep");
    mgq_status s = check_lattice(lat, false, "mgq_heatbath_sweep");
    if (s) return s;
    if ((s = check_hb_args(beta, n_hb, "mgq_heatbath_sweep"))) return s;
    for (int mu = 0; mu < 4; mu++)
        for (int par = 0; par < 2; par++)
            if ((s = heatbath_subsweep(lat, beta, sweep, n_hb, mu, par, nullptr, as_stream(stream)))) return s;
    return MGQ_OK;
}

mgq_status mgq_overrelax_sweep(mgq_lattice* lat, void* stream) {
    Trace trace("mgq_overrelax_sweep");
    mgq_status s = check_lattice(lat, false, "mgq_overrelax_sweep");
    if (s) return s;
    for (int mu = 0; mu < 4; mu++)
        for (int par = 0; par < 2; par++)
            if ((s = overrelax_subsweep(lat, mu, par, as_stream(stream)))) return s;
    return MGQ_OK;
}

mgq_status mgq_update_sweeps(mgq_lattice* lat, double beta, uint64_t sweep0, int n_sweeps, int n_hb, int n_or,
                             double* plaq_out, void* stream) {
    Trace trace("mgq_update_sweeps");
    mgq_status s = check_lattice(lat, plaq_out != nullptr, "mgq_update_sweeps");
    if (s) return s;
    if ((s = check_hb_args(beta, n_hb, "mgq_update_sweeps"))) return s;
    if (n_sweeps < 0 || n_or < 0 || n_sweeps > (int)(WS_NSCALARS - 8))
        return fail(MGQ_EINVAL, "mgq_update_sweeps: need 0 <= n_sweeps <= %d and n_or >= 0", (int)(WS_NSCALARS - 8));
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    for (int i = 0; i < n_sweeps; i++) {
        Trace sweep_trace("compound sweep");
        for (int mu = 0; mu < 4; mu++)
            for (int par = 0; par < 2; par++)
                if ((s = heatbath_subsweep(lat, beta, sweep0 + (uint64_t)i, n_hb, mu, par, nullptr, st))) return s;
        // with a plaquette record, the last overrelaxation sweep measures it
        const int n_plain = (plaq_out && n_or > 0) ? n_or - 1 : n_or;
        for (int k = 0; k < n_plain; k++)
            for (int mu = 0; mu < 4; mu++)
                for (int par = 0; par < 2; par++)
                    if ((s = overrelax_subsweep(lat, mu, par, st))) return s;
        if (plaq_out && n_or > 0 && (s = overrelax_sweep_plaquette(lat, sc + 8 + i, st))) return s;
        if (plaq_out && n_or == 0 && (s = plaquette_into(lat, ws_partials(lat), sc + 8 + i, st))) return s;
    }
    if (plaq_out) return deliver(sc + 8, plaq_out, (size_t)n_sweeps, st, "mgq_update_sweeps");
    return MGQ_OK;
}

mgq_status mgq_overrelax_sweep_plaquette(mgq_lattice* lat, double* plaq_out, void* stream) {
    Trace trace("mgq_overrelax_sweep_plaquette");
    mgq_status s = check_lattice(lat, true, "mgq_overrelax_sweep_plaquette");
    if (s) return s;
    if (!plaq_out) return fail(MGQ_EINVAL, "mgq_overrelax_sweep_plaquette: plaq_out is NULL");
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    if ((s = overrelax_sweep_plaquette(lat, sc + 5, st))) return s;
    return deliver(sc + 5, plaq_out, 1, st, "mgq_overrelax_sweep_plaquette");
}

mgq_status mgq_plaquette(const mgq_lattice* lat, double* plaq_out, void* stream) {
    Trace trace("mgq_plaquette");
    mgq_status s = check_lattice(lat, true, "mgq_plaquette");
    if (s) return s;
    if (!plaq_out) return fail(MGQ_EINVAL, "mgq_plaquette: plaq_out is NULL");
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    if ((s = plaquette_into(lat, ws_partials(lat), sc, st))) return s;
    return deliver(sc, plaq_out, 1, st, "mgq_plaquette");
}

mgq_status mgq_check_unitarity(const mgq_lattice* lat, double tol, double* max_dev_out, void* stream) {
    mgq_status s = check_lattice(lat, true, "mgq_check_unitarity");
    if (s) return s;
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    const int nb = reduction_blocks(4 * g.V, 256);
    double* sc = ws_scalars(lat);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_unitarity<T, NP><<<nb, 256, 0, st>>>(links_of<T, NP>(lat), g, ws_partials(lat));
    });
    k_final_max<<<1, 256, 0, st>>>(ws_partials(lat), nb, sc + 1);
    if ((s = cuda_check("mgq_check_unitarity"))) return s;
    double host = 0.0;
    if ((s = deliver(sc + 1, &host, 1, st, "mgq_check_unitarity"))) return s;
    if (max_dev_out) *max_dev_out = host;
    if (tol > 0.0 && host > tol) return fail(MGQ_ENONUNITARY, "mgq_check_unitarity: max deviation %.3e > %.3e", host, tol);
    return MGQ_OK;
}

}  // extern "C"
