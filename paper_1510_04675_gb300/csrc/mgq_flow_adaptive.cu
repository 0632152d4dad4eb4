// libmgq adaptive-step Wilson flow (Sec. IV.B: tolerance and maximal step as
// in Table II; the step controller follows the cited embedded Runge-Kutta
// scheme).  A trial step of size h runs the three stages of the third-order
// integrator and, from the same stage generators, the second-order solution
// W2 = exp(2 Z1 - Z0) W0.  d = max over links of |W3 - W2|_F / 3; the step is
// kept iff d <= tol and the next trial size is h min(2, 0.95 (tol/d)^(1/3)),
// capped by the maximal step and by the next measurement time.  A step that
// was cut short to land on a measurement time keeps the previous size.
//
// The controller lives on the device: each trial is a fixed sequence of
// launches whose kernels read the step size and their gate from a small
// control block, so the host never waits on a step.  It reads the finished
// flag once per chunk of trials.  The trial's kernels use programmatic
// dependent launch (see pdl_wait), so they read their predecessors' outputs
// with plain loads only.
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

struct FlowCtl {
    double t, eps, h, t_next;
    unsigned long long dbits;  // max error estimate: bits of a non-negative double
    int active;                // the current trial runs
    int hits;                  // the trial lands on the next measurement time
    int restore;               // the trial was rejected: links <- backup
    int meas;                  // measure E, Q now
    int m, steps, rejects;
    int status;                // 0 running, 1 finished, 2 step size underflow
};
static_assert(sizeof(FlowCtl) <= 16 * sizeof(double), "control block must fit 16 scalar slots");

__global__ void k_adapt_init(FlowCtl* c, double eps0) {
    c->t = 0.0;
    c->eps = eps0;
    c->h = 0.0;
    c->t_next = 0.0;
    c->dbits = 0ull;
    c->active = 0;
    c->hits = 0;
    c->restore = 0;
    c->meas = 1;  // E, Q at t = 0
    c->m = 0;
    c->steps = 0;
    c->rejects = 0;
    c->status = 0;
}

__global__ void k_adapt_begin(FlowCtl* c, double t_end, double eps_max, double dt_meas, int max_meas) {
    pdl_launch_dependents();
    pdl_wait();
    c->active = 0;
    c->restore = 0;
    c->meas = 0;
    if (c->status != 0) return;
    const double tiny = 1e-12 * dt_meas;
    if (!(c->t < t_end - tiny) || c->m >= max_meas) {
        c->status = 1;
        return;
    }
    const double t_next = fmin(dt_meas * (double)c->m, t_end);
    double h = fmin(c->eps, eps_max);
    int hits = 0;
    if (c->t + h >= t_next - tiny) {
        h = t_next - c->t;
        hits = 1;
    }
    c->t_next = t_next;
    c->h = h;
    c->hits = hits;
    c->dbits = 0ull;
    c->active = 1;
}

__global__ void k_adapt_end(FlowCtl* c, double tol, double eps_max) {
    pdl_launch_dependents();
    pdl_wait();
    if (!c->active) return;
    const double d = __longlong_as_double((long long)c->dbits);
    double fac = d > 0.0 ? 0.95 * cbrt(tol / d) : 2.0;
    if (fac > 2.0) fac = 2.0;
    if (d <= tol) {
        c->t = c->hits ? c->t_next : c->t + c->h;
        c->steps++;
        c->meas = c->hits;
        if (!c->hits) c->eps = c->h * fac;
    } else {
        c->restore = 1;
        c->rejects++;
        c->eps = c->h * fac;
        if (!(c->eps >= 1e-9 * eps_max)) c->status = 2;
    }
}

// Stage generator z = -h TA(W A(W)) coefficients, then
//   B <- aB B + cB z   (aB == 0: write only)
//   Y <- aY Y + cY z   (cY == 0: Y untouched; aY == 0: write only)
// Same 8-warp plane layout as the HMC force kernel: a block covers 32 sites in
// all eight (mu, parity) planes.
template <class T, int NP>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2)
    k_flow_stage(Links<T, NP> U, Geom g, Alg<T> B, Alg<T> Y, const FlowCtl* c, T cB, T aB, T cY, T aY) {
    pdl_launch_dependents();
    pdl_wait();
    if (!c->active) return;
    const int w = threadIdx.x >> 5;
    const int mu = w >> 1, par = w & 1;
    const int h = blockIdx.x * 32 + (threadIdx.x & 31);
    if (h >= g.Vh) return;
    int x[4];
    cb_coords(g, par, h, x);
    const M3<T> A = staple(U, g, x, h, mu, par);
    T t[8];
    ta_coeffs(mul_nn(U.load(mu, par, h), A), t);
    const T mh = (T)(-c->h);
    T* b = B.at(mu, par, h);
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const T z = mh * t[a];
        b[a * Alg<T>::kStep] = aB == T(0) ? cB * z : aB * b[a * Alg<T>::kStep] + cB * z;
    }
    if (cY != T(0)) {
        T* y = Y.at(mu, par, h);
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const T z = mh * t[a];
            y[a * Alg<T>::kStep] = aY == T(0) ? cY * z : aY * y[a * Alg<T>::kStep] + cY * z;
        }
    }
}

// W <- exp(s B) W; with backup, the old W is saved there first (the start
// of the trial, restored on rejection).
template <class T, int NP>
__global__ void __launch_bounds__(128) k_flow_exp(Links<T, NP> U, Geom g, Alg<T> B, T s, const FlowCtl* c,
                                                  Links<T, NP> backup, int save) {
    pdl_launch_dependents();
    pdl_wait();
    if (!c->active) return;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    T q[8];
    B.load(mu, par, h, q);
#pragma unroll
    for (int a = 0; a < 8; a++) q[a] *= s;
    const M3<T> u0 = U.load(mu, par, h);
    if (save) backup.store(mu, par, h, u0);
    M3<T> u = mul_nn(exp_alg(q), u0);
    if (sizeof(T) == 4) reunitarize(u);
    U.store(mu, par, h, u);
}

// d = max over links of |W3 - exp(Y) W0|_F / 3, Y = 2 Z1 - Z0.
template <class T, int NP>
__global__ void __launch_bounds__(128) k_flow_error(Links<T, NP> U, Links<T, NP> U0, Geom g, Alg<T> Y,
                                                    FlowCtl* c) {
    pdl_launch_dependents();
    pdl_wait();
    if (!c->active) return;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (idx < 8 * g.Vh) {
        const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
        T y[8];
        Y.load(mu, par, h, y);
        const M3<T> w2 = mul_nn(exp_alg(y), U0.load(mu, par, h));
        const M3<T> w3 = U.load(mu, par, h);
        // in the link precision: an FP32 estimate steers the step as well as
        // an FP64 one, and FP64 arithmetic is slow on this part
        T s2 = T(0);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const T dr = w3.e[i][j].re - w2.e[i][j].re;
                const T di = w3.e[i][j].im - w2.e[i][j].im;
                s2 += dr * dr + di * di;
            }
        d = (double)(m_sqrt(s2) / T(3));
    }
    // Non-negative doubles order like their bit patterns, and a NaN compares
    // above every number, so a broken step is rejected.
    unsigned long long bits = (unsigned long long)__double_as_longlong(d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((threadIdx.x & 31) == 0 && bits) atomicMax(&c->dbits, bits);
}

__global__ void k_flow_restore(uint4* links, const uint4* backup, size_t nwords,
                               const FlowCtl* c) {
    pdl_launch_dependents();
    pdl_wait();
    if (!c->restore) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nwords; i += (size_t)gridDim.x * blockDim.x)
        links[i] = backup[i];
}

// meas[2m] = E (site average), meas[2m+1] = Q from the clover partials; m++.
__global__ void k_adapt_meas(FlowCtl* c, const double* partials, int nb, double invV, double* meas) {
    pdl_launch_dependents();
    pdl_wait();
    if (!c->meas) return;
    double e = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        e += partials[i];
        q += partials[nb + i];
    }
    e = block_sum(e);
    q = block_sum(q);
    if (threadIdx.x == 0) {
        meas[2 * c->m] = e * invV;
        meas[2 * c->m + 1] = q;
        c->m++;
        c->meas = 0;
    }
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// Measurement times k dt_meas <= t_end, plus t_end when it is not one of them.
int adaptive_measurements(double t_end, double dt_meas) {
    const int k = (int)floor(t_end / dt_meas + 1e-9);
    return k + 1 + (t_end - k * dt_meas > 1e-12 * dt_meas ? 1 : 0);
}

}  // namespace mgq

using namespace mgq;

extern "C" {

uint64_t mgq_flow_adaptive_scratch_bytes(const mgq_lattice* lat) {
    if (!lat || !links_bytes(lat)) return 0;
    return round256(alg_bytes(lat));
}

int mgq_flow_adaptive_measurements(double t_end, double dt_meas) {
    if (!(t_end >= 0.0) || !(dt_meas > 0.0) || t_end / dt_meas > 1e6) return -1;
    return adaptive_measurements(t_end, dt_meas);
}

mgq_status mgq_wilson_flow_adaptive(mgq_lattice* lat, double t_end, double tol, double eps_max, double eps0,
                                    double dt_meas, double* E_out, double* Q_out, int* n_meas, int* n_steps,
                                    int* n_rejects, void* scratch, uint64_t scratch_bytes, void* stream) {
    Trace trace("mgq_wilson_flow_adaptive");
    mgq_status s = check_lattice(lat, true, "mgq_wilson_flow_adaptive");
    if (s) return s;
    if (!(t_end >= 0.0) || !(tol > 0.0) || !(eps_max > 0.0) || !(eps0 > 0.0) || !(dt_meas > 0.0))
        return fail(MGQ_EINVAL, "mgq_wilson_flow_adaptive: need t_end >= 0 and tol, eps_max, eps0, dt_meas > 0");
    const int nm = mgq_flow_adaptive_measurements(t_end, dt_meas);
    if (nm < 0 || 2 * nm + 32 > (int)WS_NSCALARS)
        return fail(MGQ_EINVAL, "mgq_wilson_flow_adaptive: at most %d measurements", (int)(WS_NSCALARS - 32) / 2);
    if (!scratch || ((uintptr_t)scratch & 255))
        return fail(MGQ_EINVAL, "mgq_wilson_flow_adaptive: scratch NULL or not 256-byte aligned");
    if (scratch_bytes < round256(alg_bytes(lat)))
        return fail(MGQ_ENOMEM, "mgq_wilson_flow_adaptive: scratch has %llu bytes, needs %llu",
                    (unsigned long long)scratch_bytes, (unsigned long long)round256(alg_bytes(lat)));
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    FlowCtl* c = reinterpret_cast<FlowCtl*>(sc);
    double* meas = sc + 32;
    double* partials = ws_partials(lat);
    const double invV = 1.0 / (double)g.V;
    void* Bp = ws_alg(lat);
    void* backup = ws_links(lat);
    const size_t nwords = links_bytes(lat) / 16;

    auto measure = [&]() {
        const int nb = clover_partials(lat, partials, &c->meas, st);
        launch_pdl(k_adapt_meas, 1, 512, st, c, partials, nb, invV, meas);
    };
    auto trial = [&]() {
        launch_pdl(k_adapt_begin, 1, 1, st, c, t_end, eps_max, dt_meas, nm);
        dispatch_prec(lat->prec, [&]<class T, int NP>() {
            const Links<T, NP> U = links_of<T, NP>(lat), U0 = links_at<T, NP>(backup, lat->dims);
            const Alg<T> B = alg_at<T>(Bp, lat->dims), Y = alg_at<T>(scratch, lat->dims);
            const int fb = nblk(g.Vh, 32), eb = nblk(8L * g.Vh, 128);
            // Z0: B = Z0, Y = -Z0
            launch_pdl(k_flow_stage<T, NP>, fb, 256, st, U, g, B, Y, c, T(1), T(0), T(-1), T(0));
            launch_pdl(k_flow_exp<T, NP>, eb, 128, st, U, g, B, T(0.25), c, U0, 1);
            // Z1: B = 8/9 Z1 - 17/36 B, Y = 2 Z1 + Y
            launch_pdl(k_flow_stage<T, NP>, fb, 256, st, U, g, B, Y, c, T(8.0 / 9.0), T(-17.0 / 36.0), T(2), T(1));
            launch_pdl(k_flow_exp<T, NP>, eb, 128, st, U, g, B, T(1), c, U0, 0);
            // Z2: B = 3/4 Z2 - B
            launch_pdl(k_flow_stage<T, NP>, fb, 256, st, U, g, B, Y, c, T(0.75), T(-1), T(0), T(0));
            launch_pdl(k_flow_exp<T, NP>, eb, 128, st, U, g, B, T(1), c, U0, 0);
            launch_pdl(k_flow_error<T, NP>, eb, 128, st, U, U0, g, Y, c);
        });
        launch_pdl(k_adapt_end, 1, 1, st, c, tol, eps_max);
        launch_pdl(k_flow_restore, 1184, 256, st, reinterpret_cast<uint4*>(lat->links),
                   reinterpret_cast<const uint4*>(backup), nwords, (const FlowCtl*)c);
        measure();
    };

    k_adapt_init<<<1, 1, 0, st>>>(c, eps0);
    measure();
    if ((s = cuda_check("mgq_wilson_flow_adaptive"))) return s;
    // Trials run in chunks between reads of the status word; a chunk that
    // finishes early leaves its remaining trials as gated no-op launches.
    constexpr int kChunk = 16, kMaxTrials = 1 << 20;
    int status = 0;
    for (int done = 0; status == 0; done += kChunk) {
        if (done >= kMaxTrials) return fail(MGQ_EINVAL, "mgq_wilson_flow_adaptive: more than %d trial steps", kMaxTrials);
        for (int i = 0; i < kChunk; i++) trial();
        if ((s = cuda_check("mgq_wilson_flow_adaptive"))) return s;
        if ((s = deliver_int(&c->status, &status, 1, st, "mgq_wilson_flow_adaptive"))) return s;
    }
    if (status == 2)
        return fail(MGQ_EINVAL, "mgq_wilson_flow_adaptive: step size underflow (tolerance below the precision floor)");
    int cnt[3];
    if ((s = deliver_int(&c->m, cnt, 3, st, "mgq_wilson_flow_adaptive"))) return s;
    for (int i = 0; i < cnt[0]; i++) {
        if (E_out && (s = deliver(meas + 2 * i, E_out + i, 1, st, "mgq_wilson_flow_adaptive"))) return s;
        if (Q_out && (s = deliver(meas + 2 * i + 1, Q_out + i, 1, st, "mgq_wilson_flow_adaptive"))) return s;
    }
    if (n_meas) *n_meas = cnt[0];
    if (n_steps) *n_steps = cnt[1];
    if (n_rejects) *n_rejects = cnt[2];
    return MGQ_OK;
}

}  // extern "C"
