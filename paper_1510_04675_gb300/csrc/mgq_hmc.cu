// libmgq HMC (Sec. IV.D, App. A): Gaussian su(3) momenta, the gauge force
// F = -(beta/6) TA(U A) fused with the momentum update, the exact SU(3)
// exponential link update, FP64 Hamiltonian, device-side Metropolis test and
// restore, and the PQP leapfrog driver.  The force/update kernels are shared
// with the Wilson flow (its generator is the force at beta = 6).
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// B <- alpha B + coef t(TA(U A)), t the algebra coefficients of TA(U A);
// alpha == 0 writes without reading B.  A block of 8 warps covers 32
// consecutive sites in all eight (mu, parity) planes (warp w: mu = w/2,
// parity = w%2), so the neighbour links of a site band are used by all
// directions while they are still in cache.
template <class T, int NP>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_force(Links<T, NP> U, Geom g, Alg<T> B, T coef, T alpha) {
    pdl_launch_dependents();
    const int w = threadIdx.x >> 5;
    const int mu = w >> 1, par = w & 1;
    const int h = blockIdx.x * 32 + (threadIdx.x & 31);
    int x[4];
    cb_coords(g, par, h, x);
    pdl_wait();
    if (h >= g.Vh) return;
    const M3<T> A = staple(U, g, x, h, mu, par);
    const M3<T> M = mul_nn(U.load(mu, par, h), A);
    T t[8];
    ta_coeffs(M, t);
    T* b = B.at(mu, par, h);
    if (alpha == T(0)) {
#pragma unroll
        for (int a = 0; a < 8; a++) b[a * Alg<T>::kStep] = coef * t[a];
    } else {
#pragma unroll
        for (int a = 0; a < 8; a++) b[a * Alg<T>::kStep] = alpha * b[a * Alg<T>::kStep] + coef * t[a];
    }
}

// FP32 12-real force with the staple's links staged through shared memory
// (staple_staged): a block of 4 warps covers the 4 directions of one parity for
// a 32-site band (block b: band b/2, parity b%2).
__global__ void __launch_bounds__(STAGED_THREADS, 5) k_force_staged(Links<float, 6> U, Geom g, Alg<float> B, float coef,
                                                                  float alpha) {
    extern __shared__ float4 sm[];
    pdl_launch_dependents();
    const int mu = threadIdx.x >> 5, par = blockIdx.x & 1;
    const int h = (blockIdx.x >> 1) * 32 + (threadIdx.x & 31);
    const int hc = h < g.Vh ? h : g.Vh - 1;  // lanes past the end compute a copy and store nothing
    int x[4];
    cb_coords(g, par, hc, x);
    pdl_wait();
    M3<float> u;
    // the four warps are the four directions at the same sites: U_nu(x) of the
    // upper staple terms is the updated link of warp nu
    const M3<float> A = staple_staged<NoWork, true>(U, g, x, hc, mu, par, sm, u);
    if (h >= g.Vh) return;
    const M3<float> M = mul_nn(u, A);
    float t[8];
    ta_coeffs(M, t);
    float* b = B.at(mu, par, h);
    if (alpha == 0.f) {
#pragma unroll
        for (int a = 0; a < 8; a++) b[a * Alg<float>::kStep] = coef * t[a];
    } else {
#pragma unroll
        for (int a = 0; a < 8; a++) b[a * Alg<float>::kStep] = alpha * b[a * Alg<float>::kStep] + coef * t[a];
    }
}

// U <- exp(s B) U on every link; the FP32 formats are reunitarised.
template <class T, int NP>
__global__ void __launch_bounds__(128) k_exp_update(Links<T, NP> U, Geom g, Alg<T> B, T s) {
    pdl_launch_dependents();
    pdl_wait();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    T c[8];
    B.load(mu, par, h, c);
#pragma unroll
    for (int a = 0; a < 8; a++) c[a] *= s;
    const M3<T> E = exp_alg(c);
    M3<T> u = mul_nn(E, U.load(mu, par, h));
    if (sizeof(T) == 4) reunitarize(u);
    U.store(mu, par, h, u);
}

// Gaussian momenta p_a ~ N(0,1): two draws per link, Box-Muller pairs;
// per-block partial sums of p^2/2 in FP64.
template <class T>
__global__ void __launch_bounds__(256) k_mom_refresh(Alg<T> P, Geom g, RngKey rk, double* __restrict__ partials) {
    double acc = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 8 * g.Vh; idx += gridDim.x * blockDim.x) {
        const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
        int x[4];
        cb_coords(g, par, h, x);
        const uint32_t lex = (uint32_t)lex_of(g, x);
        T p[8];
#pragma unroll
        for (int call = 0; call < 2; call++) {
            const uint4 r = draw(rk, lex, (uint32_t)mu, 0u, (uint32_t)call, KIND_MOM);
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 2; q++) {
                // Box-Muller in the momentum precision: FP64 for the parity path
                // (the oracle's momenta), FP32 otherwise (FP64 transcendentals
                // are slow on this part; the stored momenta are FP32 anyway)
                const T u0 = u01<T>(w[2 * q]), u1 = u01<T>(w[2 * q + 1]);
                const T rad = m_sqrt(T(-2) * m_log(u0));
                T sn, cs;
                sincospi(T(2) * u1, &sn, &cs);
                p[4 * call + 2 * q] = rad * cs;
                p[4 * call + 2 * q + 1] = rad * sn;
            }
        }
        P.store(mu, par, h, p);
#pragma unroll
        for (int a = 0; a < 8; a++) acc += 0.5 * (double)p[a] * (double)p[a];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <class T>
__global__ void __launch_bounds__(256) k_kinetic(Alg<T> P, Geom g, double* __restrict__ partials) {
    double acc = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 8 * g.Vh; idx += gridDim.x * blockDim.x) {
        const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
        T p[8];
        P.load(mu, par, h, p);
#pragma unroll
        for (int a = 0; a < 8; a++) acc += 0.5 * (double)p[a] * (double)p[a];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// H = kinetic + beta * 6V * (1 - plaquette), all FP64; sc[out] = H.
__global__ void k_hamiltonian(double* sc, int kin_slot, int plaq_slot, int out_slot, double beta, double nplaq) {
    sc[out_slot] = sc[kin_slot] + beta * nplaq * (1.0 - sc[plaq_slot]);
}

// dH = H1 - H0; accept iff u < exp(-dH) (u: first uniform of the accept
// draw of the trajectory), or always when accept_reject = 0.
__global__ void k_metropolis(double* sc, int h0, int h1, int dh_slot, int* flag, RngKey rk, int accept_reject) {
    const double dH = sc[h1] - sc[h0];
    sc[dh_slot] = dH;
    const uint4 r = draw(rk, 0u, 0u, 0u, 0u, KIND_ACCEPT);
    const double u = u01<double>(r.x);
    flag[0] = accept_reject ? (u < exp(-dH) ? 1 : 0) : 1;
}

// links <- backup when the trajectory was rejected (16-byte words)
__global__ void k_restore(uint4* __restrict__ links, const uint4* __restrict__ backup, size_t nwords, const int* flag) {
    if (flag[0]) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nwords; i += (size_t)gridDim.x * blockDim.x)
        links[i] = backup[i];
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// B <- alpha B + coef TA-coefficients, on `links` with the lattice's format
mgq_status force_accumulate(const mgq_lattice* lat, void* B, double coef, double alpha, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        if constexpr (sizeof(T) == 4 && NP == 6)
            launch_pdl_smem(k_force_staged, 2 * nblk(g.Vh, 32), STAGED_THREADS, STAGED_SMEM, st, links_of<T, NP>(lat), g,
                            alg_at<T>(B, lat->dims), (T)coef, (T)alpha);
        else
            launch_pdl(k_force<T, NP>, nblk(g.Vh, 32), 256, st, links_of<T, NP>(lat), g, alg_at<T>(B, lat->dims),
                       (T)coef, (T)alpha);
    });
    return cuda_check("force");
}

mgq_status exp_update(const mgq_lattice* lat, void* B, double s, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        launch_pdl(k_exp_update<T, NP>, nblk(8L * g.Vh, 128), 128, st, links_of<T, NP>(lat), g,
                   alg_at<T>(B, lat->dims), (T)s);
    });
    return cuda_check("exp_update");
}

static mgq_status kinetic_into(const mgq_lattice* lat, double* dev_out, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    const int nb = reduction_blocks(8 * g.Vh, 256);
    if (lat->prec == MGQ_F64)
        k_kinetic<double><<<nb, 256, 0, st>>>(alg_at<double>(lat->mom, lat->dims), g, ws_partials(lat));
    else
        k_kinetic<float><<<nb, 256, 0, st>>>(alg_at<float>(lat->mom, lat->dims), g, ws_partials(lat));
    launch_final_sum(ws_partials(lat), nb, 1.0, dev_out, st);
    return cuda_check("kinetic");
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_hmc_force(const mgq_lattice* lat, double beta, void* force_out, void* stream) {
    Trace trace("mgq_hmc_force");
    mgq_status s = check_lattice(lat, false, "mgq_hmc_force");
    if (s) return s;
    if (!(beta > 0.0)) return fail(MGQ_EINVAL, "mgq_hmc_force: beta must be > 0");
    if (!force_out || ((uintptr_t)force_out & 15)) return fail(MGQ_EINVAL, "mgq_hmc_force: force_out NULL or misaligned");
    return force_accumulate(lat, force_out, -beta / 6.0, 0.0, as_stream(stream));
}

mgq_status mgq_hmc_momentum_step(mgq_lattice* lat, double beta, double eps, void* stream) {
    Trace trace("mgq_hmc_momentum_step");
    mgq_status s = check_lattice(lat, false, "mgq_hmc_momentum_step");
    if (s) return s;
    if (!(beta > 0.0)) return fail(MGQ_EINVAL, "mgq_hmc_momentum_step: beta must be > 0");
    if (!(eps == eps)) return fail(MGQ_EINVAL, "mgq_hmc_momentum_step: eps is NaN");
    if (!lat->mom || ((uintptr_t)lat->mom & 15)) return fail(MGQ_EINVAL, "mgq_hmc_momentum_step: mom NULL or misaligned");
    return force_accumulate(lat, lat->mom, -eps * beta / 6.0, 1.0, as_stream(stream));
}

mgq_status mgq_link_exp_update(mgq_lattice* lat, const void* alg, double s, void* stream) {
    mgq_status st = check_lattice(lat, false, "mgq_link_exp_update");
    if (st) return st;
    if (!alg || ((uintptr_t)alg & 15)) return fail(MGQ_EINVAL, "mgq_link_exp_update: alg NULL or misaligned");
    if (!(s == s)) return fail(MGQ_EINVAL, "mgq_link_exp_update: s is NaN");
    return exp_update(lat, const_cast<void*>(alg), s, as_stream(stream));
}

mgq_status mgq_hmc_trajectory(mgq_lattice* lat, double beta, double tau, int n_steps, uint64_t traj, int accept_reject,
                              double* dH_out, int* accepted_out, void* stream) {
    Trace trace("mgq_hmc_trajectory");
    mgq_status s = check_lattice(lat, true, "mgq_hmc_trajectory");
    if (s) return s;
    if (!lat->mom) return fail(MGQ_EINVAL, "mgq_hmc_trajectory: lattice has no momentum buffer");
    if (!(beta > 0.0) || !(tau > 0.0) || n_steps < 1)
        return fail(MGQ_EINVAL, "mgq_hmc_trajectory: need beta > 0, tau > 0, n_steps >= 1");
    cudaStream_t st = as_stream(stream);
    const Geom g = make_geom(lat->dims);
    const double eps = tau / n_steps;
    const double nplaq = 6.0 * (double)g.V;
    double* sc = ws_scalars(lat);
    int* flag = reinterpret_cast<int*>(sc + 7);
    // slots: 0 kinetic, 1 plaquette, 2 H0, 3 H1, 4 dH, 7 accept flag
    const uint64_t lb = links_bytes(lat);
    if (cudaMemcpyAsync(ws_links(lat), lat->links, lb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return cuda_check("mgq_hmc_trajectory: backup");
    const RngKey rk = make_rng(lat->seed, lat->lattice_id, traj);
    const int nb = reduction_blocks(8 * g.Vh, 256);
    if (lat->prec == MGQ_F64)
        k_mom_refresh<double><<<nb, 256, 0, st>>>(alg_at<double>(lat->mom, lat->dims), g, rk, ws_partials(lat));
    else
        k_mom_refresh<float><<<nb, 256, 0, st>>>(alg_at<float>(lat->mom, lat->dims), g, rk, ws_partials(lat));
    launch_final_sum(ws_partials(lat), nb, 1.0, sc + 0, st);
    if ((s = plaquette_into(lat, ws_partials(lat), sc + 1, st))) return s;
    k_hamiltonian<<<1, 1, 0, st>>>(sc, 0, 1, 2, beta, nplaq);
    // PQP leapfrog: P(e/2) [Q(e) P(e)]^(n-1) Q(e) P(e/2)
    if ((s = force_accumulate(lat, lat->mom, -beta / 6.0 * (0.5 * eps), 1.0, st))) return s;
    for (int k = 0; k < n_steps; k++) {
        if ((s = exp_update(lat, lat->mom, eps, st))) return s;
        const double e = (k == n_steps - 1) ? 0.5 * eps : eps;
        if ((s = force_accumulate(lat, lat->mom, -beta / 6.0 * e, 1.0, st))) return s;
    }
    if ((s = kinetic_into(lat, sc + 0, st))) return s;
    if ((s = plaquette_into(lat, ws_partials(lat), sc + 1, st))) return s;
    k_hamiltonian<<<1, 1, 0, st>>>(sc, 0, 1, 3, beta, nplaq);
    k_metropolis<<<1, 1, 0, st>>>(sc, 2, 3, 4, flag, rk, accept_reject);
    k_restore<<<1184, 256, 0, st>>>(reinterpret_cast<uint4*>(lat->links), reinterpret_cast<const uint4*>(ws_links(lat)),
                                    lb / 16, flag);
    if ((s = cuda_check("mgq_hmc_trajectory"))) return s;
    if ((s = deliver(sc + 4, dH_out, dH_out ? 1 : 0, st, "mgq_hmc_trajectory"))) return s;
    return deliver_int(flag, accepted_out, accepted_out ? 1 : 0, st, "mgq_hmc_trajectory");
}

}  // extern "C"
