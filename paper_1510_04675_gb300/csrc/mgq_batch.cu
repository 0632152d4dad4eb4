// libmgq batched driver: many independent lattices of (possibly) different
// extents, couplings and RNG streams advanced together -- the parallel
// rethermalisation of N_s prolongated configurations (Sec. II: "embarrassingly
// parallel").  Each sub-sweep is ONE launch over all lattices: the grid is a
// flattened list of 128-site blocks, block b belongs to the lattice l with
// prefix[l] <= b < prefix[l+1].  The lattice descriptors travel as kernel
// parameters (no device-side table), so a whole call can be captured into a
// CUDA graph as is.
#include <cstring>

#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

constexpr int BATCH_CHUNK = 128;  // lattices per launch (kernel-parameter table)
constexpr int BATCH_THREADS = 128;     // the kernels' maximal block size
constexpr int BATCH_MIN_THREADS = 32;  // the smallest tunable block size (sizes the partial sums)

template <class T>
struct LatDesc {
    Cx<T>* links;
    Geom g;
    T beta;
    uint2 key;
};

template <class T>
struct Batch {
    int n;
    int prefix[BATCH_CHUNK + 1];  // block offsets
    LatDesc<T> d[BATCH_CHUNK];
};

template <class T>
__device__ __forceinline__ int find_lattice(const Batch<T>& B, int b) {
    int lo = 0, hi = B.n;  // prefix[lo] <= b < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (B.prefix[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

template <class T>
__device__ __forceinline__ const Geom& geom_of(const LatDesc<T>& d) {
    return d.g;
}

// The staple of U_MU(x) and the link itself: staged through shared memory for
// FP32 12-real links (staple_staged; the launch gives STAGED_THREADS threads and
// STAGED_SMEM bytes), as in the single-lattice kernels, so that batched and
// single-lattice updates agree bit for bit; plain loads otherwise.
template <class T, int NP, int MU>
__device__ __forceinline__ void staple_and_link(const Links<T, NP>& U, const Geom& g, const int x[4], int h, int par,
                                                M3<T>& A, M3<T>& u) {
    if constexpr (sizeof(T) == 4 && NP == 6) {
        extern __shared__ float4 staged_sm[];
        A = staple_staged(U, g, x, h, MU, par, staged_sm, u);
    } else {
        A = staple(U, g, x, h, MU, par);
        u = U.load(MU, par, h);
    }
}

// NHB1: single-attempt instance (the attempt loop is removed at compile time)
template <class T, int NP, int MU, bool NHB1>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(T) == 8 ? 2 : 4)
    k_heatbath_batched(const __grid_constant__ Batch<T> B, int par, uint32_t idx_lo, uint32_t idx_hi, int n_hb) {
    if constexpr (NHB1) n_hb = 1;
    pdl_launch_dependents();
    const int l = find_lattice(B, blockIdx.x);
    const LatDesc<T>& d = B.d[l];
    const int h = (blockIdx.x - B.prefix[l]) * (int)blockDim.x + threadIdx.x;
    pdl_wait();
    if (h >= d.g.Vh) return;
    const Geom g = geom_of(d);
    Links<T, NP> U;
    U.p = d.links;
    U.S = d.g.S;
    RngKey rk;
    rk.key = d.key;
    rk.idx_lo = idx_lo;
    rk.idx_hi = idx_hi;
    int x[4];
    cb_coords(g, par, h, x);
    M3<T> A, u;
    staple_and_link<T, NP, MU>(U, g, x, h, par, A, u);
    hb_link(u, A, d.beta, n_hb, rk, (uint32_t)lex_of(g, x), (uint32_t)MU, (uint8_t*)nullptr);
    U.store(MU, par, h, u);
}

template <class T, int NP, int MU>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(T) == 8 ? 2 : 4) k_overrelax_batched(const __grid_constant__ Batch<T> B, int par) {
    pdl_launch_dependents();
    const int l = find_lattice(B, blockIdx.x);
    const LatDesc<T>& d = B.d[l];
    const int h = (blockIdx.x - B.prefix[l]) * (int)blockDim.x + threadIdx.x;
    pdl_wait();
    if (h >= d.g.Vh) return;
    const Geom g = geom_of(d);
    Links<T, NP> U;
    U.p = d.links;
    U.S = d.g.S;
    int x[4];
    cb_coords(g, par, h, x);
    M3<T> A, u;
    staple_and_link<T, NP, MU>(U, g, x, h, par, A, u);
    or_link(u, A);
    U.store(MU, par, h, u);
}

// The last overrelaxation sweep's direction-3 sub-sweeps with the plaquette
// folded in, as in the single-lattice driver: partial sums per block at
// partials[par * nblocks + blockIdx.x].
template <class T, int NP>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(T) == 8 ? 2 : 4)
    k_overrelax_batched_last(const __grid_constant__ Batch<T> B, int par, double* __restrict__ partials) {
    pdl_launch_dependents();
    const int l = find_lattice(B, blockIdx.x);
    const LatDesc<T>& d = B.d[l];
    const int h = (blockIdx.x - B.prefix[l]) * (int)blockDim.x + threadIdx.x;
    pdl_wait();
    double acc = 0.0;
    if (h < d.g.Vh) {
        const Geom g = geom_of(d);
        Links<T, NP> U;
        U.p = d.links;
        U.S = d.g.S;
        int x[4];
        cb_coords(g, par, h, x);
        M3<T> A, u;
        staple_and_link<T, NP, 3>(U, g, x, h, par, A, u);
        if (par == 1) acc = (double)retr_nn(u, A);
        or_link(u, A);
        U.store(3, par, h, u);
        acc += site_plaquettes<T, NP, 3>(U, g, par, h);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[par * B.prefix[B.n] + blockIdx.x] = acc;
}

// one block per lattice: both parities' partials of its blocks, times 1/(18 V)
template <class T>
__global__ void k_overrelax_batched_last_final(const __grid_constant__ Batch<T> B, const double* __restrict__ partials,
                                               double* __restrict__ out) {
    const int l = blockIdx.x, nb = B.prefix[B.n];
    double v = 0.0;
    for (int i = B.prefix[l] + threadIdx.x; i < B.prefix[l + 1]; i += blockDim.x) v += partials[i] + partials[nb + i];
    v = block_sum(v);
    if (threadIdx.x == 0) out[l] = v / (18.0 * (double)B.d[l].g.V);
}

// per-lattice plaquette: blocks of 256 sites, partial sums at the global block index
template <class T, int NP>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_plaquette_batched(const __grid_constant__ Batch<T> B, double* __restrict__ partials) {
    const int l = find_lattice(B, blockIdx.x);
    const LatDesc<T>& d = B.d[l];
    const int idx = (blockIdx.x - B.prefix[l]) * 256 + threadIdx.x;
    double acc = 0.0;
    if (idx < d.g.V) {
        Links<T, NP> U;
        U.p = d.links;
        U.S = d.g.S;
        const int par = idx >= d.g.Vh, h = idx - par * d.g.Vh;
        acc = site_plaquettes(U, geom_of(d), par, h);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// one block per lattice: fixed-order sum of its partials, times 1/(18 V)
template <class T>
__global__ void k_plaquette_batched_final(const __grid_constant__ Batch<T> B, const double* __restrict__ partials,
                                          double* __restrict__ out) {
    const int l = blockIdx.x;
    double v = 0.0;
    for (int i = B.prefix[l] + threadIdx.x; i < B.prefix[l + 1]; i += blockDim.x) v += partials[i];
    v = block_sum(v);
    if (threadIdx.x == 0) out[l] = v / (18.0 * (double)B.d[l].g.V);
}

template <class T>
static void fill_batch(Batch<T>& B, const mgq_lattice* lats, const double* betas, int first, int n, int sites_per_block,
                       bool half) {
    B.n = n;
    B.prefix[0] = 0;
    for (int i = 0; i < n; i++) {
        const mgq_lattice& L = lats[first + i];
        const Geom g = make_geom(L.dims);
        LatDesc<T>& d = B.d[i];
        d.links = reinterpret_cast<Cx<T>*>(L.links);
        d.g = g;
        d.beta = betas ? (T)betas[first + i] : T(1);
        const RngKey rk = make_rng(L.seed, L.lattice_id, 0);
        d.key = rk.key;
        const int units = half ? g.Vh : g.V;
        B.prefix[i + 1] = B.prefix[i] + (units + sites_per_block - 1) / sites_per_block;
    }
}

// partial-sum slots: two per 128-site half-lattice block (the plaquette-
// measuring overrelaxation sub-sweeps), which also covers one per 256-site
// block (the plaquette kernel)
uint64_t batch_partials(const mgq_lattice* lats, int n) {
    uint64_t nb = 0;
    for (int i = 0; i < n; i++) {
        const Geom g = make_geom(lats[i].dims);
        nb += 2 * (uint64_t)((g.Vh + BATCH_MIN_THREADS - 1) / BATCH_MIN_THREADS);
    }
    return nb;
}

}  // namespace mgq

using namespace mgq;

extern "C" {

uint64_t mgq_batch_workspace_bytes(const mgq_lattice* lats, int n_lat, int n_sweeps) {
    if (!lats || n_lat < 1 || n_sweeps < 0) return 0;
    for (int i = 0; i < n_lat; i++)
        if (!valid_dims(lats[i].dims)) return 0;
    return round256(batch_partials(lats, n_lat) * sizeof(double)) + round256((uint64_t)n_sweeps * n_lat * sizeof(double));
}

mgq_status mgq_update_sweeps_batched(mgq_lattice* lats, int n_lat, const double* betas, uint64_t sweep0, int n_sweeps,
                                     int n_hb, int n_or, double* plaq_out, void* batch_work, uint64_t batch_work_bytes,
                                     void* stream) {
    Trace trace("mgq_update_sweeps_batched");
    if (!lats || n_lat < 1) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: need at least one lattice");
    if (!betas) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: betas is NULL");
    mgq_status s;
    for (int i = 0; i < n_lat; i++) {
        if ((s = check_lattice(&lats[i], false, "mgq_update_sweeps_batched"))) return s;
        if (lats[i].prec != lats[0].prec) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: all lattices need one precision");
        if (!(betas[i] > 0.0) || betas[i] > 1e6) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: beta[%d] invalid", i);
    }
    if (n_hb < 1 || n_hb > 256) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: n_hb must be in [1, 256]");
    if (n_sweeps < 0 || n_or < 0) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: negative counts");
    const uint64_t need = mgq_batch_workspace_bytes(lats, n_lat, n_sweeps);
    if (plaq_out) {
        if (!batch_work) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: plaquettes need batch_work");
        if (((uintptr_t)batch_work & 255) != 0) return fail(MGQ_EINVAL, "mgq_update_sweeps_batched: batch_work not 256-byte aligned");
        if (batch_work_bytes < need)
            return fail(MGQ_ENOMEM, "mgq_update_sweeps_batched: batch_work has %llu bytes, needs %llu",
                        (unsigned long long)batch_work_bytes, (unsigned long long)need);
    }
    cudaStream_t st = as_stream(stream);
    double* partials = reinterpret_cast<double*>(batch_work);
    double* results =
        plaq_out ? reinterpret_cast<double*>((char*)batch_work + round256(batch_partials(lats, n_lat) * sizeof(double)))
                 : nullptr;
    for (int i = 0; i < n_sweeps; i++) {
        const uint64_t sweep = sweep0 + (uint64_t)i;
        for (int first = 0; first < n_lat; first += BATCH_CHUNK) {
            const int n = (n_lat - first < BATCH_CHUNK) ? n_lat - first : BATCH_CHUNK;
            dispatch_prec(lats[0].prec, [&]<class T, int NP>() {
                const bool staged = sizeof(T) == 4 && NP == 6;
                const int bh = staged ? STAGED_THREADS : block_size(MGQ_KERNEL_HEATBATH_BATCHED, lats[0].prec);
                const int bo = staged ? STAGED_THREADS : block_size(MGQ_KERNEL_OVERRELAX_BATCHED, lats[0].prec);
                const size_t smem = staged ? (size_t)STAGED_SMEM : 0;
                Batch<T> Bl, Bo;
                fill_batch(Bl, lats, betas, first, n, bh, true);
                fill_batch(Bo, lats, betas, first, n, bo, true);
                const int nblocks = Bl.prefix[n], oblocks = Bo.prefix[n];
                for (int mu = 0; mu < 4; mu++)
                    for (int par = 0; par < 2; par++)
                        dispatch_mu(mu, [&]<int MU>() {
                            if (n_hb == 1)
                                launch_pdl_smem(k_heatbath_batched<T, NP, MU, true>, nblocks, bh, smem, st, Bl, par,
                                           (uint32_t)(sweep & 0xffffffffu), (uint32_t)(sweep >> 32), n_hb);
                            else
                                launch_pdl_smem(k_heatbath_batched<T, NP, MU, false>, nblocks, bh, smem, st, Bl, par,
                                           (uint32_t)(sweep & 0xffffffffu), (uint32_t)(sweep >> 32), n_hb);
                        });
                // with a plaquette record, the last overrelaxation sweep's
                // direction-3 sub-sweeps measure it (per-chunk partials)
                const bool fold = plaq_out && n_or > 0;
                for (int k = 0; k < n_or; k++)
                    for (int mu = 0; mu < 4; mu++)
                        for (int par = 0; par < 2; par++) {
                            if (fold && k == n_or - 1 && mu == 3) {
                                launch_pdl_smem(k_overrelax_batched_last<T, NP>, oblocks, bo, smem, st, Bo, par, partials);
                                continue;
                            }
                            dispatch_mu(mu, [&]<int MU>() {
                                launch_pdl_smem(k_overrelax_batched<T, NP, MU>, oblocks, bo, smem, st, Bo, par);
                            });
                        }
                if (fold)
                    k_overrelax_batched_last_final<T><<<n, 256, 0, st>>>(Bo, partials,
                                                                         results + (size_t)i * n_lat + first);
            });
            if ((s = cuda_check("mgq_update_sweeps_batched"))) return s;
        }
        if (plaq_out && n_or == 0) {
            uint64_t poff = 0;
            for (int first = 0; first < n_lat; first += BATCH_CHUNK) {
                const int n = (n_lat - first < BATCH_CHUNK) ? n_lat - first : BATCH_CHUNK;
                dispatch_prec(lats[0].prec, [&]<class T, int NP>() {
                    Batch<T> Bl;
                    fill_batch(Bl, lats, betas, first, n, 256, false);
                    k_plaquette_batched<T, NP><<<Bl.prefix[n], 256, 0, st>>>(Bl, partials + poff);
                    k_plaquette_batched_final<T><<<n, 256, 0, st>>>(Bl, partials + poff, results + (size_t)i * n_lat + first);
                    poff += (uint64_t)Bl.prefix[n];
                });
            }
            if ((s = cuda_check("mgq_update_sweeps_batched: plaquette"))) return s;
        }
    }
    if (plaq_out) return deliver(results, plaq_out, (size_t)n_sweeps * n_lat, st, "mgq_update_sweeps_batched");
    return MGQ_OK;
}

}  // extern "C"
