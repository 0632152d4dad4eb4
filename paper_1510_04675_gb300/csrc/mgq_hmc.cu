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

// FP32 12-real force with the staple's links staged through shared memory (the
// cp.async pipeline of staple_staged): a block of 4 warps covers the 4
// directions of one parity for a 32-site band (block b: band b/2, parity b%2),
// so warp mu, lane l holds U_mu(x) of the band's site l.
//
// Each of the six plaquettes at x is formed once.  The upper term of U_mu(x) in
// plane nu, U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ = P_mu,nu(x), is the
// adjoint of the upper term of U_nu(x) in plane mu, and TA(M^+) = -TA(M) with TA
// linear, so
//   TA(U_mu A_mu) = TA(U_mu A_mu^dn) + sum_{nu owned} TA(P_mu,nu) - sum_{nu other} TA(P_nu,mu)
// where A^dn holds the three lower terms.  The owner of plane {mu, nu} is warp mu
// when nu = mu + 1 (mod 4), or nu = mu + 2 with mu < 2: warp 0 forms P_01 and
// P_02, warp 1 P_12 and P_13, warp 2 P_23, warp 3 P_30.  Owners leave their TA
// coefficients in shared memory; the partner warp subtracts them after a
// barrier.  Per site this is 12 lower and 6 upper staple terms where the plain
// staple takes 12 of each.  The half-terms run lower first, then the owned
// upper ones; U_nu(x) of an upper term is the updated link warp nu staged.
//
// Shared memory per thread column (STAGED_SMEM in all): two stages of three
// staged links, the updated link in slot (2, 0); its row 2 is published in slot
// (0, 2), which the upper terms leave free, and the TA coefficients of owned
// plane j in slot (1, j) once stage 1 has no more terms to stage.
__device__ __forceinline__ void staged_ta_store(float4* sm, int j, const float t[8]) {
    *staged_slot(sm, 1, j, 0) = make_float4(t[0], t[1], t[2], t[3]);
    *staged_slot(sm, 1, j, 1) = make_float4(t[4], t[5], t[6], t[7]);
}
__device__ __forceinline__ void staged_ta_sub(const float4* sm, int col, int j, float t[8]) {
    const float4 a = sm[((1 * 3 + j) * 3 + 0) * STAGED_THREADS + col];
    const float4 b = sm[((1 * 3 + j) * 3 + 1) * STAGED_THREADS + col];
    t[0] -= a.x, t[1] -= a.y, t[2] -= a.z, t[3] -= a.w;
    t[4] -= b.x, t[5] -= b.y, t[6] -= b.z, t[7] -= b.w;
}

__global__ void __launch_bounds__(STAGED_THREADS, 5) k_force_staged(Links<float, 6> U, Geom g, Alg<float> B, float coef,
                                                                  float alpha) {
    extern __shared__ float4 sm[];
    pdl_launch_dependents();
    const int mu = threadIdx.x >> 5, par = blockIdx.x & 1, op = par ^ 1, lane = threadIdx.x & 31;
    const int h = (blockIdx.x >> 1) * 32 + lane;
    const int hc = h < g.Vh ? h : g.Vh - 1;  // lanes past the end compute a copy and store nothing
    const int n_own = mu < 2 ? 2 : 1;       // owned planes: nu = mu + 1, mu + 2 (mod 4)
    const int n_terms = 3 + n_own;
    int x[4];
    cb_coords(g, par, hc, x);
    const Hops H = make_hops(g, x);
    const int fmu = pick(H.fwd, mu);
    const int hpm = (H.lex + fmu) >> 1;
    int hmn[3], hpm_mn[3], nus[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int nu = i < mu ? i : i + 1;
        nus[i] = nu;
        hmn[i] = (H.lex + pick(H.bwd, nu)) >> 1;
        hpm_mn[i] = (H.lex + fmu + pick(H.bwd, nu)) >> 1;
    }
    int own_nu[2], own_hpn[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
        own_nu[j] = (mu + 1 + j) & 3;
        own_hpn[j] = (H.lex + pick(H.fwd, own_nu[j])) >> 1;
    }
    pdl_wait();
    // half-term k < 3: dn = (e d)^+ f, d = U_nu(x+mu-nu), e = U_mu(x-nu), f = U_nu(x-nu)
    // for the k-th direction nu != mu; k >= 3: up = (a b^+) c^+ for owned plane
    // j = k - 3, a = U_nu(x+mu), b = U_mu(x+nu), c = U_nu(x) (shared)
    auto issue = [&](int k, int stage) {
        if (k < 3) {
            stage_link(sm, stage, 0, U, nus[k], par, hpm_mn[k]);
            stage_link(sm, stage, 1, U, mu, op, hmn[k]);
            stage_link(sm, stage, 2, U, nus[k], op, hmn[k]);
        } else {
            stage_link(sm, stage, 0, U, own_nu[k - 3], op, hpm);
            stage_link(sm, stage, 1, U, mu, op, own_hpn[k - 3]);
        }
    };
    stage_link(sm, 2, 0, U, mu, par, hc);  // the updated link, with the first half-term
    issue(0, 0);
    cp_async_commit();
    issue(1, 1);
    cp_async_commit();
    M3<float> A;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A.e[i][j] = mk(0.f, 0.f);
    M3<float> u;
    float t[8];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        if (k >= n_terms) break;
        if (k + 1 < n_terms) cp_async_wait<1>();
        else cp_async_wait<0>();
        const int st = k & 1;
        if (k < 3) {
            M3<float> d = mul_nn_2(staged_rows(sm, st, 1), staged_full(sm, st, 0));
            rebuild_row2(d);
            M3<float> term = mul_dn_2(d, staged_full(sm, st, 2));
            rebuild_row2(term);
            acc_add(A, term);
        } else {
            const int j = k - 3;
            const M3<float> ab = mul_nd_2(staged_rows(sm, st, 0), staged_full(sm, st, 1));
            M3<float> up = mul_nd_2(ab, own_full_of(sm, own_nu[j] * 32 + lane));
            rebuild_row2(up);
            M3<float> P = mul_nn_2(u, up);
            rebuild_row2(P);
            float tp[8];
            ta_coeffs(P, tp);
#pragma unroll
            for (int a = 0; a < 8; a++) t[a] += tp[a];
            staged_ta_store(sm, j, tp);  // stage 1 stages nothing after term 3
        }
        if (k + 2 < n_terms) {
            issue(k + 2, st);
            cp_async_commit();
        }
        if (k == 2) {
            // the lower terms are done: complete the updated link, publish its
            // row 2 in the slot the upper terms leave free, and take TA(U A^dn)
            u = staged_full(sm, 2, 0);
            *staged_slot(sm, 0, 2, 0) = make_float4(u.e[2][0].re, u.e[2][0].im, u.e[2][1].re, u.e[2][1].im);
            *reinterpret_cast<float2*>(staged_slot(sm, 0, 2, 1)) = make_float2(u.e[2][2].re, u.e[2][2].im);
            ta_coeffs(mul_nn(u, A), t);
            __syncthreads();  // every warp's updated link is staged and completed
        }
    }
    __syncthreads();  // every owner's TA coefficients are in shared memory
    // planes owned by another warp: nu = mu - 1 (its first owned plane) and,
    // for mu >= 2, nu = mu - 2 (its second)
    staged_ta_sub(sm, ((mu + 3) & 3) * 32 + lane, 0, t);
    if (mu >= 2) staged_ta_sub(sm, (mu - 2) * 32 + lane, 1, t);
    if (h >= g.Vh) return;
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
