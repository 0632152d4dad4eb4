/*
 * mgq.h -- C ABI of libmgq, the GB300 (sm_103a) hot path of the multiscale
 * thermalization of pure SU(3) Yang-Mills theory (Endres, Brower, Detmold,
 * Orginos, Pochinsky, "Multiscale Monte Carlo equilibration: Pure Yang-Mills
 * theory", arXiv:1510.04675).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Ownership: the caller allocates every buffer (links, momenta, workspace,
 *   outputs) and keeps it alive until the work queued on `stream` is done.
 *   The library allocates no device memory.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *   work is queued asynchronously on it.  An entry point that writes a
 *   result to a HOST pointer synchronises `stream` before returning; output
 *   pointers may be host or device memory and are classified with
 *   cudaPointerGetAttributes.
 * Errors: every entry point returns an mgq_status and never aborts; the
 *   message of the last failure on the calling thread is mgq_last_error().
 *   Argument errors are detected before any work is queued.
 * Lattice (Sec. III): D = 4 hypercube with extents dims[0..3] (all even,
 *   >= 2), periodic boundary conditions, V = dims[0]*dims[1]*dims[2]*dims[3]
 *   <= 2^28 sites (128^4; 51.5 GB of links in the 12-real FP32 format).  Site (x0,x1,x2,x3) has lexicographic index
 *   x0 + L0*(x1 + L1*(x2 + L2*x3)) and parity (x0+x1+x2+x3) mod 2.
 *
 * Device link layout (owned by the caller, written by the library)
 * ----------------------------------------------------------------
 *   links[mu][parity][h/32][plane][h%32], mu = 0..3, parity = 0..1,
 *   h = lex/2 in 0..V/2-1, site stride S = mgq_site_stride(dims) >= V/2 (a
 *   multiple of 64): per (mu, parity), S/32 blocks of 32 consecutive sites,
 *   each holding plane 0 of its 32 sites, then plane 1, and so on.
 *   Each element of a plane is one complex number of the link matrix U_mu(x)
 *   (re, im adjacent):
 *     MGQ_F64     : 9 planes (row-major 3x3) of double2   -> 144 B per link
 *     MGQ_F32     : 9 planes of float2                     ->  72 B per link
 *     MGQ_F32_C12 : 6 planes (rows 0 and 1) of float2; row 2 is rebuilt as
 *                   conj(row0 x row1) on every load        ->  48 B per link
 *   Momenta / Lie-algebra fields: mom[mu][parity][h/32][a][h%32], a = 0..7, the
 *   coefficients p_a of P = sum_a p_a X_a, X_a = i lambda_a / 2 (Gell-Mann),
 *   as double (MGQ_F64) or float (MGQ_F32, MGQ_F32_C12).
 *
 * Canonical exchange layout (mgq_import_links / mgq_export_links): double
 *   canon[V][4][3][3][2], site lexicographic, then mu, row, column, re/im.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *   counter = (site_lex, mu | subgroup<<2 | attempt<<4 | kind<<12,
 *              lo32(index), hi32(index)),
 *   key = (lo32(seed), hi32(seed) ^ lattice_id); kind 1 = heat bath,
 *   2 = hot start, 3 = momenta, 4 = HMC accept; index = sweep or trajectory.
 *   Results therefore depend only on (seed, lattice_id, index), not on the
 *   launch configuration.
 */
#ifndef MGQ_H
#define MGQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGQ_ABI_VERSION 1

typedef enum {
    MGQ_OK = 0,
    MGQ_EINVAL = 1,         /* invalid argument (message in mgq_last_error)       */
    MGQ_ENOMEM = 2,         /* caller-provided workspace too small                */
    MGQ_ECUDA = 3,          /* a CUDA runtime call or kernel launch failed        */
    MGQ_EUNSUPPORTED = 4,   /* valid request outside the built scope (e.g. open BC) */
    MGQ_ETIMEOUT = 5,       /* a bounded device wait gave up                      */
    MGQ_ENONUNITARY = 6     /* mgq_check_unitarity found a link off SU(3)         */
} mgq_status;

typedef enum { MGQ_F64 = 0, MGQ_F32 = 1, MGQ_F32_C12 = 2 } mgq_prec;
typedef enum { MGQ_WILSON = 0 } mgq_action;               /* the paper's action (Sec. III) */
typedef enum { MGQ_PERIODIC = 0, MGQ_OPEN = 1 } mgq_bc;   /* periodic only (Sec. IV.A)    */

/* One lattice and the caller's device buffers for it. */
typedef struct mgq_lattice {
    int32_t dims[4];       /* L0..L3, each even and >= 2; product <= 2^28          */
    int32_t bc[4];         /* mgq_bc per direction; only MGQ_PERIODIC is supported */
    int32_t prec;          /* mgq_prec: storage and arithmetic format of the links */
    int32_t action;        /* mgq_action                                           */
    uint64_t seed;         /* Philox key, low and high words                       */
    uint32_t lattice_id;   /* xor-ed into the key's high word: one stream per lattice */
    uint32_t reserved;     /* must be 0                                            */
    void* links;           /* device, mgq_links_bytes() bytes                       */
    void* mom;             /* device, mgq_mom_bytes() bytes; HMC only, else NULL   */
    void* work;            /* device, >= mgq_workspace_bytes() bytes, 256-B aligned */
    uint64_t work_bytes;   /* size of `work`                                       */
} mgq_lattice;

/* ---- sizes and diagnostics ------------------------------------------------ */
int mgq_abi_version(void);
const char* mgq_status_string(mgq_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* mgq_last_error(void);
/* Per-parity site stride S (elements) for the given extents; 0 if invalid. */
uint64_t mgq_site_stride(const int32_t dims[4]);
/* Bytes of the link array, the momentum array and the workspace for `lat`
 * (only dims and prec are read); 0 if the extents or precision are invalid. */
uint64_t mgq_links_bytes(const mgq_lattice* lat);
uint64_t mgq_mom_bytes(const mgq_lattice* lat);
uint64_t mgq_workspace_bytes(const mgq_lattice* lat);

/* ---- launch tuning ------------------------------------------------------------
 * Threads per block, per storage format, of the checkerboard sub-sweep kernels
 * (heat bath and overrelaxation) of the single-lattice and the batched entry
 * points and of the APE step of the prolongation: 32, 64, 96 or 128 (the
 * kernels are compiled for at most 128); 128 by default.  Results do not
 * depend on it (one thread per link or per active bond).  FP32 12-real
 * sub-sweeps of the batched driver, and of single lattices with V/2 >= 49152,
 * stage their staple links through shared memory and always run 128 threads
 * per block; the setting applies to the other launches.  The force kernel's shape is structural (eight warps cover the
 * eight (mu, parity) planes of a 32-site band) and not tuned.  Process-wide setting; change it only while no
 * call is being issued.  Set by the autotuner (paper_1510_04675_gb300/tune.py). */
typedef enum {
    MGQ_KERNEL_HEATBATH = 0,
    MGQ_KERNEL_OVERRELAX = 1,
    MGQ_KERNEL_HEATBATH_BATCHED = 2,
    MGQ_KERNEL_OVERRELAX_BATCHED = 3,
    MGQ_KERNEL_APE = 4
} mgq_kernel;
mgq_status mgq_set_block_size(int kernel, int prec, int threads);
/* Current value, 0 for an unknown kernel or precision. */
int mgq_get_block_size(int kernel, int prec);

/* FP32 arithmetic probe: one launch of independent packed FP32 FMA chains on
 * every SM (4 blocks of 256 threads per SM, `iters` iterations of 16 packed
 * FMAs per thread); *sink (device, 4 bytes) receives a value that depends on
 * every chain.  Returns the number of floating-point operations the launch
 * performs (2 per FMA), 0 on a bad argument; time it with events on `stream`
 * to measure the FP32 peak that the ALU-bound kernels are compared with. */
uint64_t mgq_fma_probe(int iters, float* sink, void* stream);

/* ---- fields ---------------------------------------------------------------- */
/* Start configurations (Sec. IV.E): start = 0 cold (unit links, the ordered
 * delta-function start), start = 1 hot (Haar-random SU(3) per link from the
 * hot-start Philox stream).  Errors: MGQ_EINVAL. */
mgq_status mgq_init_links(mgq_lattice* lat, int start, void* stream);

/* Project every link back onto SU(3) with the Gram-Schmidt reunitarisation the
 * update kernels apply after each link update (rows 0, 1 normalised and
 * orthogonalised, row 2 = conj(row0 x row1); the paper is silent on it).  For
 * FP32 formats fp64_projection = 1 runs the projection in FP64 and rounds the
 * result to FP32, 0 runs it in FP32; FP64 fields ignore the flag.
 * Errors: MGQ_EINVAL. */
mgq_status mgq_reunitarize(mgq_lattice* lat, int fp64_projection, void* stream);

/* Copy a field between the canonical FP64 layout (device pointer `canon`,
 * V*4*18 doubles) and the lattice's own layout.  Import rounds to the
 * lattice precision (MGQ_F32_C12 keeps rows 0 and 1); export rebuilds
 * row 2 for MGQ_F32_C12.  Errors: MGQ_EINVAL, MGQ_ECUDA. */
mgq_status mgq_import_links(mgq_lattice* lat, const double* canon, void* stream);
mgq_status mgq_export_links(const mgq_lattice* lat, double* canon, void* stream);

/* ---- local updates (Sec. IV.A: Cabibbo-Marinari heat bath with Creutz's
 *      SU(2) sampler, Brown-Woch overrelaxation, checkerboard schedule) ---- */

/* One heat-bath sweep at coupling beta (Sec. III: beta = 2 Nc / g^2): for
 * mu = 0..3, parity = 0, 1, every link U_mu(x) of that subset is updated
 * from its staple: V = U A, for the subgroups (0,1), (0,2), (1,2) up to n_hb
 * Creutz attempts (1 <= n_hb <= 256), U <- R U, then Gram-Schmidt
 * reunitarisation.  `sweep` is the RNG index.  Errors: MGQ_EINVAL. */
mgq_status mgq_heatbath_sweep(mgq_lattice* lat, double beta, uint64_t sweep, int n_hb, void* stream);

/* One (mu, parity) subset of the sweep above.  decisions (device, optional,
 * uint8[V][4][3] in lexicographic site order) receives for each updated link
 * and subgroup the accepted attempt index, or 255 if none was accepted. */
mgq_status mgq_heatbath_subsweep(mgq_lattice* lat, double beta, uint64_t sweep, int n_hb, int mu,
                                 int parity, uint8_t* decisions, void* stream);

/* One overrelaxation sweep (same schedule; per subgroup the reflection
 * R = (w/|w|)^2 that keeps Re Tr(U A) unchanged).  No RNG, no beta. */
mgq_status mgq_overrelax_sweep(mgq_lattice* lat, void* stream);

/* One overrelaxation sweep, as mgq_overrelax_sweep, that also returns the
 * average plaquette of the field it leaves (as mgq_plaquette, to rounding):
 * the two sub-sweeps of direction 3 that end the sweep measure it on the fly
 * (Sec. IV.A; the paper's plaquette record, Sec. III), so no separate pass
 * reads the links.  plaq_out: one double, host or device.  Needs the
 * workspace (it uses the algebra buffer for per-block sums).  mgq_update_sweeps
 * uses it for the last overrelaxation sweep of each compound sweep when it
 * records plaquettes.  Errors: MGQ_EINVAL, MGQ_ENOMEM. */
mgq_status mgq_overrelax_sweep_plaquette(mgq_lattice* lat, double* plaq_out, void* stream);

/* n_sweeps compound sweeps, each 1 heat-bath sweep (RNG index sweep0 + i)
 * followed by n_or overrelaxation sweeps (Sec. IV.A uses n_or = 10; the
 * benchmarked configurations use 4).  plaq_out (optional, n_sweeps doubles,
 * host or device) receives the average plaquette after each compound sweep. */
mgq_status mgq_update_sweeps(mgq_lattice* lat, double beta, uint64_t sweep0, int n_sweeps, int n_hb,
                             int n_or, double* plaq_out, void* stream);

/* ---- batched driver (Sec. II: the N_s prolongated configurations are
 *      rethermalised independently, "embarrassingly parallel") ------------- */

/* Bytes of caller workspace `batch_work` needed by mgq_update_sweeps_batched
 * for n_lat lattices and n_sweeps plaquette records; 0 on invalid extents. */
uint64_t mgq_batch_workspace_bytes(const mgq_lattice* lats, int n_lat, int n_sweeps);

/* mgq_update_sweeps for n_lat independent lattices at once: each may have its
 * own extents, coupling betas[l] (host array), seed and lattice_id; all share
 * one precision and the sweep indices sweep0 + i.  Every sub-sweep is one
 * launch over all lattices (descriptors passed by value, at most 128 lattices
 * per launch), so the call can be captured into a CUDA graph.  Results are
 * bit-identical to n_lat separate mgq_update_sweeps calls.  plaq_out
 * (optional, host or device, n_sweeps x n_lat doubles, sweep-major) receives
 * every lattice's FP64 average plaquette after each compound sweep (measured
 * by the last overrelaxation sweep, as in mgq_update_sweeps) and then
 * needs batch_work (device, 256-B aligned, >= mgq_batch_workspace_bytes).
 * Errors: MGQ_EINVAL (no lattice: n_lat < 1; mixed precision, bad beta, ...),
 * MGQ_ENOMEM. */
mgq_status mgq_update_sweeps_batched(mgq_lattice* lats, int n_lat, const double* betas, uint64_t sweep0,
                                     int n_sweeps, int n_hb, int n_or, double* plaq_out, void* batch_work,
                                     uint64_t batch_work_bytes, void* stream);

/* ---- observables (Sec. III, IV.B-C) ----------------------------------------- */

/* Average plaquette (1/(6V)) sum_x sum_{mu<nu} (1/3) Re Tr U_munu(x),
 * accumulated in FP64.  plaq_out: one double, host or device. */
mgq_status mgq_plaquette(const mgq_lattice* lat, double* plaq_out, void* stream);

/* The same average plaquette for callers that cannot give the library any
 * device memory (for example code running under another framework's memory
 * manager that owns the device memory and forbids further cudaMalloc, or a
 * latency-critical monitoring hook where cudaMalloc/cudaFree would implicitly
 * synchronise the device).  The paper has no counterpart: this is a library
 * convenience.  It ignores lat->work and allocates nothing; its scratch is a
 * fixed 64 KiB static device array inside libmgq that every GPU loading the
 * library holds until exit.  Limit: V <= 2,096,896 sites (one partial sum per
 * 256 sites, 8191 slots; e.g. 32^4 fits, 48^4 does not); larger lattices get
 * MGQ_EINVAL and should use mgq_plaquette.  Every call outside stream capture
 * looks up the array's device address (cudaGetSymbolAddress) with the calling
 * device current, so a context re-created after cudaDeviceReset is followed;
 * a call under stream capture reuses the address of the last call outside
 * capture on that device, so make a first call before any capture (a captured
 * call with no such address returns MGQ_EINVAL), and none after a device
 * reset without a call outside capture in between.  All calls share
 * the one array and it keeps the last call's contents (each call rewrites
 * every slot it reads), so calls that overlap on the GPU -- concurrent
 * streams, or other host threads on the same device -- race and must be
 * serialised by the caller.  plaq_out: one double, host or device. */
mgq_status mgq_plaquette_noalloc(const mgq_lattice* lat, double* plaq_out, void* stream);

/* Space-time averaged m x n Wilson loop (Sec. III):
 * (1/(6V)) sum_x sum_{mu<nu} (1/3) Re Tr L^m_mu(x) L^n_nu(x+m mu)
 * L^m_mu(x+n nu)^+ L^n_nu(x)^+, with the Wilson lines L^m_mu the ordered
 * products of m links; 1 <= m, n <= 64.  out: one double, host or device. */
mgq_status mgq_wilson_loop(const mgq_lattice* lat, int m, int n, double* out, void* stream);

/* Rethermalisation diagnostics (Sec. III, IV.C, IV.E), nine doubles (host or
 * device): out[0..2] partial plaquettes W^{1x1}_d (plaquettes with
 * chi_munu(n) = d, normalised by N^{1x1}_d = 2 (D-d)(D-d-1) C(D,d) N_0/2^D),
 * out[3..7] displaced loops W^{2x2}_d (2x2 loops from sites with chi(n) = d,
 * N^{2x2}_d = C(D,2) C(D,d) N_0/2^D), out[8] h = max_p N_c [1 - W^{1x1}_p]
 * (admissibility when h < 0.067). */
mgq_status mgq_partial_loops(const mgq_lattice* lat, double* out, void* stream);

/* Clover energy density E = (1/V) sum_x -1/2 sum_{mu,nu} Tr G_munu^2 and
 * charge Q = -1/(32 pi^2) sum_x eps_{munurhosigma} Tr G_munu G_rhosigma,
 * G_munu = traceless part of (Q_munu - Q_munu^+)/8 (four clover leaves).
 * E_out, Q_out: one double each (either may be NULL), host or device. */
mgq_status mgq_topo_charge(const mgq_lattice* lat, double* E_out, double* Q_out, void* stream);

/* Three-loop improved topological charge (Sec. IV.C, the gluonic operator of
 * de Forcrand, Garcia Perez and Stamatescu, Nucl. Phys. B 499 (1997) 409):
 * Q_m = sum_x q_m(x) with q_m the clover density above built from the four
 * m x m leaves of every plane (m = 1, 2, 3), and
 * Q = 3/2 Q_1 - 3/5 Q_2 / 2^4 + 1/10 Q_3 / 3^4, the tree-level coefficients
 * that cancel the O(a^2) and O(a^4) terms of the m x m clovers.
 * Q_out[4] = {Q, Q_1, Q_2, Q_3} (host or device).  Needs the workspace.
 * Errors: MGQ_EINVAL, MGQ_ENOMEM. */
mgq_status mgq_topo_charge_improved(const mgq_lattice* lat, double* Q_out, void* stream);

/* Wilson flow with fixed step eps (Sec. IV.B), Luscher's third-order
 * Runge-Kutta scheme with generator Z(W) = -TA(W A(W)); n_steps steps, the
 * links are replaced by the flowed field.  E and Q (as mgq_topo_charge) are
 * measured at t = k eps for k = 0, meas_every, 2 meas_every, ... <= n_steps:
 * E_out, Q_out hold n_steps/meas_every + 1 doubles (host or device, NULL to
 * skip).  Uses the workspace's algebra buffer.  Errors: MGQ_EINVAL, MGQ_ENOMEM. */
mgq_status mgq_wilson_flow(mgq_lattice* lat, double eps, int n_steps, int meas_every, double* E_out,
                           double* Q_out, void* stream);

/* Wilson flow to t_end in the form of the problem statement: fixed steps of
 * size eps (Sec. IV.B, the RK3 step above), except that a step that would pass
 * the next measurement time, or t_end, is shortened to end on it.  E (clover)
 * and Q are measured at the n_meas flow times t_meas[] (host, ascending, each
 * in [0, t_end]; at most 224) into E_out[i], Q_out[i] (host or device, NULL to
 * skip).  charge 0: clover Q; charge 1: the three-loop improved Q of
 * mgq_topo_charge_improved (Sec. IV.C).  The links are replaced by the field
 * at t_end.  Uses the workspace's algebra buffer.  Errors: MGQ_EINVAL (bad
 * times, eps <= 0, more than 1e8 steps), MGQ_ENOMEM. */
mgq_status mgq_wilson_flow_times(mgq_lattice* lat, double t_end, double eps, const double* t_meas, int n_meas,
                                 int charge, double* E_out, double* Q_out, void* stream);

/* Adaptive-step Wilson flow (Sec. IV.B, Table II: tolerance 0.01, maximal
 * step 0.2, measurements every t0/4).  Each trial step of size h runs the
 * three stages above and the embedded second-order solution
 * W2 = exp(2 Z1 - Z0) W0; d = max over links of |W3 - W2|_F / 3.  The step is
 * kept iff d <= tol; the next trial size is h min(2, 0.95 (tol/d)^(1/3)),
 * capped by eps_max and by the next measurement time k dt_meas (a step cut
 * short there keeps the previous size).  eps0 is the first trial size.  The
 * links are replaced by the field flowed to t_end.  E and Q are measured at
 * t = k dt_meas <= t_end and at t_end: E_out, Q_out hold
 * mgq_flow_adaptive_measurements(t_end, dt_meas) doubles (host or device, NULL
 * to skip); n_meas, n_steps, n_rejects (host, NULL to skip) receive the
 * measurements made, the accepted steps and the rejected trials.  The step
 * control runs on the device; the call synchronises `stream` once per 16
 * trials and therefore cannot be captured into a CUDA graph.  scratch: device,
 * 256-byte aligned, >= mgq_flow_adaptive_scratch_bytes.  Uses the workspace's
 * link copy and algebra buffer.  Errors: MGQ_EINVAL (bad arguments, more than
 * 240 measurements, step size underflow when tol is below the precision's
 * rounding floor, more than 2^20 trials), MGQ_ENOMEM. */
mgq_status mgq_wilson_flow_adaptive(mgq_lattice* lat, double t_end, double tol, double eps_max, double eps0,
                                    double dt_meas, double* E_out, double* Q_out, int* n_meas, int* n_steps,
                                    int* n_rejects, void* scratch, uint64_t scratch_bytes, void* stream);

/* Bytes of the scratch of mgq_wilson_flow_adaptive (one algebra field); 0 on
 * invalid extents or precision. */
uint64_t mgq_flow_adaptive_scratch_bytes(const mgq_lattice* lat);

/* Number of measurements of mgq_wilson_flow_adaptive: the times k dt_meas <=
 * t_end plus t_end when it is not one of them; -1 on invalid arguments. */
int mgq_flow_adaptive_measurements(double t_end, double dt_meas);

/* ---- adjoint Wilson flow (reverse mode through the RK3 step above) ------------
 * Cotangents are algebra fields in the mom layout and precision; a cotangent
 * L at a field W pairs with the variation W_l -> exp(e_l) W_l as
 * sum_l sum_a L_l,a e_l,a. */

/* Bytes of the caller scratch of mgq_wilson_flow_step_adjoint (2 link fields
 * + 7 algebra fields); 0 on invalid extents or precision. */
uint64_t mgq_flow_adjoint_scratch_bytes(const mgq_lattice* lat);

/* g_out = J(omega)^T g_in: pulls a cotangent g_in at the field exp(omega) U back
 * to the algebra variable omega, J(X)^T = sum_n (-ad_X)^n / (n+1)! the adjoint
 * of the differential of exp (d/dt e^{X + tY} e^{-X} = sum_n ad_X^n Y/(n+1)!).
 * With it a function of exp(omega) U gets its true omega-derivative, not only
 * the Lie derivative at omega = 0 (the exponential of the HMC Q-step, Sec. IV.D,
 * and of every RK3 stage, Sec. IV.B, have this differential).  omega, g_in,
 * g_out: device algebra fields in the mom layout and precision (g_in may equal
 * g_out).  Errors: MGQ_EINVAL (NULL or misaligned pointers, bad lattice). */
mgq_status mgq_exp_vjp(const mgq_lattice* lat, const void* omega, const void* g_in, void* g_out, void* stream);

/* lambda += scale * DZ(W)^T [psi]: the vector-Jacobian product of the flow
 * generator Z(W) = -TA(W A(W)) at W = lat->links (all device, mom layout). */
mgq_status mgq_flow_vjp(const mgq_lattice* lat, const void* psi, double scale, void* lambda, void* stream);

/* One step of the adjoint flow: on entry `lambda` is a cotangent at
 * Phi_eps(W0), the field one RK3 step of size eps after W0 = lat->links; on
 * return it is the pulled-back cotangent at W0.  W0 is not modified; the
 * step's intermediate fields are recomputed into `scratch` (device, 256-B
 * aligned, >= mgq_flow_adjoint_scratch_bytes).  Errors: MGQ_EINVAL,
 * MGQ_ENOMEM. */
mgq_status mgq_wilson_flow_step_adjoint(const mgq_lattice* lat, double eps, void* lambda, void* scratch,
                                        uint64_t scratch_bytes, void* stream);

/* Bytes of the caller scratch of mgq_clover_vjp (6 planes x 8 reals per site). */
uint64_t mgq_clover_vjp_scratch_bytes(const mgq_lattice* lat);

/* lambda += scale * dO/de: the gradient of the clover observable O
 * (observable 0: E, 1: Q, as in mgq_topo_charge) with respect to the links
 * at lat->links, as a cotangent (mom layout and precision, device).  This is
 * the starting cotangent of the backward pass of a flowed clover observable.
 * scratch: device, 256-B aligned, >= mgq_clover_vjp_scratch_bytes.
 * Errors: MGQ_EINVAL, MGQ_ENOMEM. */
mgq_status mgq_clover_vjp(const mgq_lattice* lat, int observable, double scale, void* lambda, void* scratch,
                          uint64_t scratch_bytes, void* stream);

/* ---- HMC (Sec. IV.D, App. A) ------------------------------------------------- */

/* Gauge force F(x,mu) = -(beta/6) TA(U_mu(x) A_mu(x)) into force_out
 * (device, mom layout and precision); dP/dt = F for H = sum p^2/2 + S. */
mgq_status mgq_hmc_force(const mgq_lattice* lat, double beta, void* force_out, void* stream);

/* The P-step of the leapfrog (Sec. IV.D), force fused with the update:
 * P_mu(x) <- P_mu(x) + eps F(x,mu) on lat->mom, F as in mgq_hmc_force -- the
 * kernel the trajectory runs (eps = e/2 or e).  One pass reads every link and
 * reads and writes P.  Errors: MGQ_EINVAL (mom NULL or misaligned, beta <= 0). */
mgq_status mgq_hmc_momentum_step(mgq_lattice* lat, double beta, double eps, void* stream);

/* The Q-step of the leapfrog (Sec. IV.D): U_mu(x) <- exp(s P_mu(x)) U_mu(x)
 * on every link, P = sum_a p_a X_a read from `alg` (device, mom layout and
 * precision), exact SU(3) exponential (Cayley-Hamilton form of Morningstar
 * and Peardon); FP32 formats are reunitarised.  Errors: MGQ_EINVAL. */
mgq_status mgq_link_exp_update(mgq_lattice* lat, const void* alg, double s, void* stream);

/* One unit-length-style trajectory of length tau with n_steps PQP leapfrog
 * steps: Gaussian momenta from the momentum stream of `traj` into lat->mom,
 * H0 = sum p^2/2 + S (FP64), P(e/2) [Q(e) P(e)]^(n-1) Q(e) P(e/2) with
 * Q(e): U <- exp(e P) U, H1, dH = H1 - H0 (FP64); accept iff u < exp(-dH)
 * with u from the accept stream of `traj`; accept_reject = 0 accepts
 * unconditionally (warm-up trajectories, Sec. IV.E).  A rejection restores
 * the links from the workspace copy.  dH_out / accepted_out: one double /
 * one int, host or device, either may be NULL.  Needs lat->mom.
 * Errors: MGQ_EINVAL, MGQ_ENOMEM. */
mgq_status mgq_hmc_trajectory(mgq_lattice* lat, double beta, double tau, int n_steps, uint64_t traj,
                              int accept_reject, double* dH_out, int* accepted_out, void* stream);

/* ---- multiscale maps (Sec. III: Eqs. restriction, prolongation, smoothing,
 *      APE) ------------------------------------------------------------------ */

/* Prolongation of `coarse` onto `fine` (fine dims = 2 x coarse dims, same
 * precision): transfer U^f_mu(n) = U^c_mu(n/2), U^f_mu(n+e_mu) = 1 at chi(n)
 * = 0 and 1 elsewhere; then for d = 0, 1, 2 Jacobi APE steps
 * U <- P_SU(3)[U + c sum_{nu: n_nu odd} (T+ + T-)] on the bonds with
 * chi_mu(n) = d + 1 until |S_d(k) - S_d(k-1)| <= rel_tol |S_d(k-1)| or
 * max_iter steps (rel_tol <= 0: exactly max_iter steps).  The stopping rule
 * and the stage changes run on the device (Sec. IV.C's 0.001 % rule is
 * rel_tol = 1e-5); the host reads a finished flag every 32 APE iterations.
 * iters_out (3 ints) and sd_out (3 doubles), host or device, NULL to skip,
 * receive the steps taken and the final S_d / beta.  Uses fine->work.
 * Errors: MGQ_EINVAL, MGQ_ENOMEM. */
mgq_status mgq_prolongate(const mgq_lattice* coarse, mgq_lattice* fine, double c, double rel_tol,
                          int max_iter, int* iters_out, double* sd_out, void* stream);

/* Bytes of the work buffer of mgq_prolongate_batched for these fine lattices:
 * the per-lattice stage state and partial sums, and one scratch link field per
 * lattice; 0 on invalid extents or precision. */
uint64_t mgq_prolongate_batched_workspace_bytes(const mgq_lattice* fine, int n);

/* Prolongation (as mgq_prolongate) of n independent lattices of possibly
 * different extents at once -- the N_s configurations refined in parallel
 * (Sec. II) -- each with its own stage, step count and stopping decision on
 * the device.  Every APE iteration is one launch per 64 lattices; a stage
 * of k steps takes k + 1 iterations, so a lattice whose stages take k0, k1, k2
 * steps is finished after k0 + k1 + k2 + 3 iterations, and later iterations
 * leave it alone.  iter_budget = 0: iterate until every lattice finished (the
 * host reads the finished count every 32 iterations).  iter_budget > 0: run
 * exactly that many iterations and never synchronise, so the call can be
 * captured into a CUDA graph; lattices not finished by then keep their newest
 * field and report the steps of their current stage.  iters_out (3n ints),
 * sd_out (3n doubles) and n_done_out (the number of finished lattices, 1 int):
 * host or device, NULL to skip (a host pointer synchronises the stream).
 * work: device, 256-byte aligned, >= mgq_prolongate_batched_workspace_bytes.
 * Errors: MGQ_EINVAL (no pair: n < 1; extents, precisions, ...), MGQ_ENOMEM. */
mgq_status mgq_prolongate_batched(const mgq_lattice* coarse, mgq_lattice* fine, int n, double c, double rel_tol,
                                  int max_iter, int iter_budget, int* iters_out, double* sd_out, int* n_done_out,
                                  void* work, uint64_t work_bytes, void* stream);

/* Restriction U^c_mu(n/2) = U^f_mu(n) U^f_mu(n + e_mu) at chi(n) = 0. */
mgq_status mgq_restrict(const mgq_lattice* fine, mgq_lattice* coarse, void* stream);

/* ---- checks ------------------------------------------------------------------ */
/* max over links of max(|U U^+ - 1|, |det U - 1|) into max_dev_out (one
 * HOST double, may be NULL); synchronises `stream`.  Returns MGQ_ENONUNITARY
 * when the deviation exceeds tol (> 0).  Uses the workspace. */
mgq_status mgq_check_unitarity(const mgq_lattice* lat, double tol, double* max_dev_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MGQ_H */
