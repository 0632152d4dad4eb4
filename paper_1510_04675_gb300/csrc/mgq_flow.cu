// libmgq Wilson flow (Sec. IV.B; fixed step, Luscher's third-order
// Runge-Kutta integrator) and clover observables E(t), Q(t) (Sec. IV.B-C).
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

mgq_status force_accumulate(const mgq_lattice* lat, void* B, double coef, double alpha, cudaStream_t st);
mgq_status exp_update(const mgq_lattice* lat, void* B, double s, cudaStream_t st);

// Per site: E(x) = -1/2 sum_{mu,nu} Tr G^2 = 1/2 sum_{mu<nu} |g_munu|^2 and
// q(x) = -1/(32 pi^2) eps Tr(G G) = 1/(8 pi^2) (g01.g23 - g02.g13 + g03.g12),
// using Tr(X_a X_b) = -delta_ab / 2.
template <class T, int NP>
__global__ void __launch_bounds__(128) k_clover(Links<T, NP> U, Geom g, double* __restrict__ partials,
                                               const int* __restrict__ gate) {
    if (gate && !__ldg(gate)) return;  // grid-uniform: the whole launch skips
    double e = 0.0, q = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        int x[4];
        cb_coords(g, par, h, x);
        T G[6][8];
        const int pl[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
#pragma unroll 1
        for (int p = 0; p < 6; p++) clover_coeffs(U, g, x, par, h, pl[p][0], pl[p][1], G[p]);
        // per-site sums in the link precision (FP64 arithmetic is slow on this
        // part), accumulated over sites in FP64
        T es = T(0), d01_23 = T(0), d02_13 = T(0), d03_12 = T(0);
#pragma unroll
        for (int a = 0; a < 8; a++) {
#pragma unroll
            for (int p = 0; p < 6; p++) es += G[p][a] * G[p][a];
            d01_23 += G[0][a] * G[5][a];
            d02_13 += G[1][a] * G[4][a];
            d03_12 += G[2][a] * G[3][a];
        }
        e += 0.5 * (double)es;
        q += ((double)d01_23 - (double)d02_13 + (double)d03_12) * (1.0 / (8.0 * 9.869604401089358));
    }
    e = block_sum(e);
    q = block_sum(q);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = e;
        partials[gridDim.x + blockIdx.x] = q;
    }
}

int clover_partials(const mgq_lattice* lat, double* partials, const int* gate, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    const int nb = reduction_blocks(g.V, 128) < 2048 ? reduction_blocks(g.V, 128) : 2048;
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_clover<T, NP><<<nb, 128, 0, st>>>(links_of<T, NP>(lat), g, partials, gate);
    });
    return nb;
}

mgq_status clover_into(const mgq_lattice* lat, double* partials, double* dev_out, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    const int nb = clover_partials(lat, partials, nullptr, st);
    launch_final_sum(partials, nb, 1.0 / (double)g.V, dev_out, st);
    launch_final_sum(partials + nb, nb, 1.0, dev_out + 1, st);
    return cuda_check("clover");
}

mgq_status improved_charge_into(const mgq_lattice* lat, double* partials, double* dev_out, cudaStream_t st);

// One RK3 step of size eps with the workspace's algebra buffer B:
// Z_i = eps Z(W_i), Z(W) = -TA(W A(W));
// W1 = exp(Z0/4) W0; W2 = exp(8/9 Z1 - 17/36 Z0) W1; W3 = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2
static mgq_status flow_step(mgq_lattice* lat, void* B, double eps, cudaStream_t st) {
    mgq_status s;
    if ((s = force_accumulate(lat, B, -eps, 0.0, st))) return s;                       // B = Z0
    if ((s = exp_update(lat, B, 0.25, st))) return s;
    if ((s = force_accumulate(lat, B, -eps * 8.0 / 9.0, -17.0 / 36.0, st))) return s;  // B = 8/9 Z1 - 17/36 Z0
    if ((s = exp_update(lat, B, 1.0, st))) return s;
    if ((s = force_accumulate(lat, B, -eps * 0.75, -1.0, st))) return s;               // B = 3/4 Z2 - B
    return exp_update(lat, B, 1.0, st);
}

// E and Q of the current links into meas[0], meas[1] (device); charge 1 takes
// the three-loop improved Q (its four values pass through tmp[0..3]).
static mgq_status measure_EQ(const mgq_lattice* lat, int charge, double* meas, double* tmp, cudaStream_t st) {
    mgq_status s = clover_into(lat, ws_partials(lat), meas, st);
    if (s || !charge) return s;
    if ((s = improved_charge_into(lat, ws_partials(lat), tmp, st))) return s;
    if (cudaMemcpyAsync(meas + 1, tmp, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return cuda_check("measure_EQ");
    return MGQ_OK;
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_topo_charge(const mgq_lattice* lat, double* E_out, double* Q_out, void* stream) {
    Trace trace("mgq_topo_charge");
    mgq_status s = check_lattice(lat, true, "mgq_topo_charge");
    if (s) return s;
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    if ((s = clover_into(lat, ws_partials(lat), sc + 16, st))) return s;
    if ((s = deliver(sc + 16, E_out, E_out ? 1 : 0, st, "mgq_topo_charge"))) return s;
    return deliver(sc + 17, Q_out, Q_out ? 1 : 0, st, "mgq_topo_charge");
}

mgq_status mgq_wilson_flow(mgq_lattice* lat, double eps, int n_steps, int meas_every, double* E_out, double* Q_out,
                           void* stream) {
    Trace trace("mgq_wilson_flow");
    mgq_status s = check_lattice(lat, true, "mgq_wilson_flow");
    if (s) return s;
    if (!(eps > 0.0) || n_steps < 0 || meas_every < 1)
        return fail(MGQ_EINVAL, "mgq_wilson_flow: need eps > 0, n_steps >= 0, meas_every >= 1");
    const int nm = n_steps / meas_every + 1;
    if (2 * nm + 32 > (int)WS_NSCALARS) return fail(MGQ_EINVAL, "mgq_wilson_flow: at most %d measurements", (int)(WS_NSCALARS - 32) / 2);
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    double* meas = sc + 32;  // E at meas[2m], Q at meas[2m+1]
    void* B = ws_alg(lat);
    int m = 0;
    for (int k = 0; k <= n_steps; k++) {
        if (k % meas_every == 0) {
            if ((s = clover_into(lat, ws_partials(lat), meas + 2 * m, st))) return s;
            m++;
        }
        if (k == n_steps) break;
        if ((s = flow_step(lat, B, eps, st))) return s;
    }
    // gather strided E, Q pairs
    for (int i = 0; i < nm; i++) {
        if (E_out && (s = deliver(meas + 2 * i, E_out + i, 1, st, "mgq_wilson_flow"))) return s;
        if (Q_out && (s = deliver(meas + 2 * i + 1, Q_out + i, 1, st, "mgq_wilson_flow"))) return s;
    }
    return MGQ_OK;
}

mgq_status mgq_wilson_flow_times(mgq_lattice* lat, double t_end, double eps, const double* t_meas, int n_meas,
                                 int charge, double* E_out, double* Q_out, void* stream) {
    Trace trace("mgq_wilson_flow_times");
    mgq_status s = check_lattice(lat, true, "mgq_wilson_flow_times");
    if (s) return s;
    if (!(eps > 0.0) || !(t_end >= 0.0) || n_meas < 0 || (n_meas > 0 && !t_meas) || charge < 0 || charge > 1)
        return fail(MGQ_EINVAL, "mgq_wilson_flow_times: need eps > 0, t_end >= 0, n_meas >= 0, t_meas, charge 0 or 1");
    if (2 * n_meas + 64 > (int)WS_NSCALARS)
        return fail(MGQ_EINVAL, "mgq_wilson_flow_times: at most %d measurements", (int)(WS_NSCALARS - 64) / 2);
    for (int i = 0; i < n_meas; i++)
        if (!(t_meas[i] >= 0.0) || t_meas[i] > t_end || (i > 0 && t_meas[i] < t_meas[i - 1]))
            return fail(MGQ_EINVAL, "mgq_wilson_flow_times: t_meas must be ascending within [0, t_end]");
    if (t_end / eps > 1e8) return fail(MGQ_EINVAL, "mgq_wilson_flow_times: more than 1e8 steps");
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    double* meas = sc + 64;  // E at meas[2i], Q at meas[2i+1]
    void* B = ws_alg(lat);
    const double tiny = 1e-12 * (t_end > 1.0 ? t_end : 1.0);
    double t = 0.0;
    int i = 0;
    while (i < n_meas && t_meas[i] <= t + tiny) {
        if ((s = measure_EQ(lat, charge, meas + 2 * i, sc + 24, st))) return s;
        i++;
    }
    while (t < t_end - tiny) {
        // the next stop: the next measurement time below t_end, else t_end
        const double stop = (i < n_meas && t_meas[i] < t_end) ? t_meas[i] : t_end;
        const double h = stop - t < eps ? stop - t : eps;
        if ((s = flow_step(lat, B, h, st))) return s;
        t = h == stop - t ? stop : t + h;
        while (i < n_meas && t_meas[i] <= t + tiny) {
            if ((s = measure_EQ(lat, charge, meas + 2 * i, sc + 24, st))) return s;
            i++;
        }
    }
    for (int k = 0; k < n_meas; k++) {
        if (E_out && (s = deliver(meas + 2 * k, E_out + k, 1, st, "mgq_wilson_flow_times"))) return s;
        if (Q_out && (s = deliver(meas + 2 * k + 1, Q_out + k, 1, st, "mgq_wilson_flow_times"))) return s;
    }
    return MGQ_OK;
}

}  // extern "C"
