/*
 * sgw.h -- C ABI of the GB300 (sm_103a) stochastic-GW hot path.
 *
 * The library computes the data-parallel core of stochastic GW in the sROI form:
 * batched Chebyshev filtering and propagation of stochastic orbitals on a periodic
 * real-space grid, the linear-response time-dependent-Hartree (TDH) step, the time
 * ordering of the induced potential, the zeta propagation with the Sigma_c(t)
 * accumulation, and the transform of Sigma to frequency and the QP solve.
 *
 * Conventions (all entry points):
 *  - Grids are cubic, n^3 points with spacing h (bohr); n in {16, 32, 64, 128} (plane path: one
 *    xy plane per CTA, two HBM passes per H application) or n in {48, 96, 288} (row path:
 *    n = 2^a 3^b, units of 8 x rows per CTA plus y- and z-line passes, four HBM passes per H
 *    application; the 288^2 plane does not fit one CTA's shared memory).  Results agree between
 *    the paths to FP32 rounding; the split-operator entries need the plane path (SGW_EINVAL).
 *    A grid function is stored with x fastest: index g = (z*n + y)*n + x.
 *  - A complex vector is interleaved complex64 ("c64": float re, float im), N_g
 *    elements; a batch of B vectors is B contiguous vectors [B][N_g].
 *  - The inner product is <a|b> = dV sum_g conj(a_g) b_g, dV = h^3.
 *  - Hartree atomic units throughout.
 *  - Pointers named *_dev are device pointers on the context's device; *_host are
 *    host pointers.  The caller owns every input and output buffer; the library
 *    owns only what the context allocates (plans, tables, projector data, scratch).
 *  - Calls are asynchronous on the context's stream unless stated; those that
 *    return host scalars synchronise that stream before returning.
 *  - No call throws or aborts.  Errors are returned as an sgw_status; the message
 *    of the last error is available from sgw_last_error().  A device-side failure
 *    detected by a kernel (e.g. a bounded wait that ran out) is reported as
 *    SGW_ETIMEOUT or SGW_ECUDA by the next synchronising call.
 *  - Device buffers must be 16-byte aligned (cudaMalloc / torch allocations are).
 */
#ifndef SGW_H
#define SGW_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgw_ctx sgw_ctx;

typedef enum {
    SGW_OK = 0,
    SGW_EINVAL = 1,    /* bad argument (size, pointer, unsupported grid) */
    SGW_ENOMEM = 2,    /* device or host allocation failed */
    SGW_ECUDA = 3,     /* a CUDA runtime call failed */
    SGW_ESTATE = 4,    /* call out of order (e.g. no potential set yet) */
    SGW_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    SGW_ENOCONV = 6    /* no root of the QP equation in the search window */
} sgw_status;

/* Library version string (static storage). */
const char* sgw_version(void);

/* Message of the last error on this context (static per context; NULL ctx gives the
 * last error of sgw_setup_grid). */
const char* sgw_last_error(const sgw_ctx* ctx);

/*
 * Create a context for an n^3 periodic grid of spacing h.
 * Sec. 2.2: H is applied on a Fourier grid, FFT pairs switching between the position
 * and momentum representations.  ecut > 0 enables the kinetic-energy cutoff of Sec. 2.2
 * / Table 2 read as T(k) = min(|k|^2/2, ecut); ecut <= 0 disables it.
 * max_batch: the largest number of vectors any later call will pass (sizes scratch:
 * 3 * max_batch * N_g * 8 bytes).  stream: a cudaStream_t (NULL = default stream).
 * device: CUDA device ordinal (made current for every call on this context).
 */
sgw_status sgw_setup_grid(sgw_ctx** out, int nx, int ny, int nz, double h, double ecut,
                          int max_batch, int device, void* stream);

/* Release the context and everything it allocated. */
void sgw_destroy(sgw_ctx* ctx);

/* Replace the stream used by later calls. */
sgw_status sgw_set_stream(sgw_ctx* ctx, void* stream);

/*
 * Graph mode (enable != 0): sgw_filter_occupied, sgw_propagate, sgw_tdh_response and sgw_sigma_c
 * capture their whole launch sequence (every Chebyshev term of every time step) into a CUDA graph
 * on their first call with a given set of arguments and buffers, and replay the instantiated graph
 * on later calls with the same ones (up to 8 cached graphs per context; the cache is dropped when
 * the potential, the stream or a work area changes).  Results are identical to direct launches.
 * Needs a non-default stream; ignored on the default stream and while profiling is enabled.
 * Such calls must not themselves be made inside a caller's stream capture.
 */
sgw_status sgw_set_graph_mode(sgw_ctx* ctx, int enable);

/*
 * Launch tuning (the paper's GPU port batches all vectors of a step into each launch, Sec. 2.3;
 * these keys refine how those launches use the memory system).  Every key is a performance hint:
 * no result depends on it.
 *   SGW_TUNE_PLANE_OPERANDS   : bit 0 (1) = each xy-plane pass block starts by prefetching into L2
 *                               the operands of its pointwise step (b_{k+1}, psi, b_{k+2},
 *                               potential rows), so they arrive while its inverse transform runs;
 *                               bit 1 (2, the 288 grid's 36-row step only) = b_{k+1}, psi, b_{k+2}
 *                               are read and the step's outputs written with evict-first
 *                               (streaming) caching, so that they do not displace prefetched or
 *                               shared lines in L2; values 0-3 (default 1)
 *   SGW_TUNE_PLANE_LOOKAHEAD  : each xy-plane pass block also prefetches into L2 the input plane of
 *                               the block this many blocks later in launch order (0 = off, default)
 *   SGW_TUNE_PENCIL_LOOKAHEAD : the same for the z-pencil pass, in pencil blocks (0 = off, default)
 *   SGW_TUNE_PLANE_VARIANT    : form of the xy-plane pass: 0 = one block of n^2/16 threads per plane
 *                               (default), 1 = twice as many threads (one butterfly per thread per
 *                               FFT stage), 2 = persistent blocks that walk their planes and copy the
 *                               next plane's input into a second shared-memory buffer (cp.async)
 *                               while the current one is transformed (n <= 64; at n = 128 it runs
 *                               as 0); at n = 288: 0 = row form (passes over y lines and over
 *                               36-row units, default), 1 = one thread-block cluster of 8 CTAs
 *                               per xy plane with 32 warps per CTA, 2 = the same with 18 warps
 *   SGW_TUNE_LINE_FORM        : form of the line passes on the 288 grid: 0 = z lines on tiles of
 *                               16 kx-columns transformed by radix stages in shared memory with the
 *                               first and last stages in registers (default), 1 = the same with 32
 *                               columns, 2 = tiles of 16 columns with one warp FFT per column;
 *                               3 = the z lines and the row form's y lines by a two-stage
 *                               16 x 18 transform (one shared-memory round trip per transform),
 *                               4 = form 3 with the 36-row step's rows transformed the same way
 *                               instead of by warp FFTs.  Forms 0-2 leave the y lines on radix
 *                               stages.
 * On row-path grids (n = 48, 96, 288) the other keys are accepted and have no effect, and the
 * autotuner keeps their current values; SGW_TUNE_PLANE_VARIANT, SGW_TUNE_LINE_FORM and
 * SGW_TUNE_PLANE_OPERANDS (for the row form's 36-row step) act at n = 288.
 * sgw_set_tuning returns SGW_EINVAL for an unknown key or a negative value (a value above 3 for
 * SGW_TUNE_PLANE_OPERANDS, above 2 for SGW_TUNE_PLANE_VARIANT, above 4 for SGW_TUNE_LINE_FORM) and drops the context's cached graphs; sgw_get_tuning writes the current
 * value to *value_host.
 */
enum {
    SGW_TUNE_PLANE_OPERANDS = 0,
    SGW_TUNE_PLANE_LOOKAHEAD = 1,
    SGW_TUNE_PENCIL_LOOKAHEAD = 2,
    SGW_TUNE_PLANE_VARIANT = 3,
    SGW_TUNE_LINE_FORM = 4,
    SGW_TUNE_KEYS = 5
};
sgw_status sgw_set_tuning(sgw_ctx* ctx, int key, int value);
sgw_status sgw_get_tuning(sgw_ctx* ctx, int key, int* value_host);

/*
 * Autotuner: time `reps` degree-8 Chebyshev sums (the propagator's two-pass term, KB included when
 * a KB part is set) on a scratch batch of `batch` vectors for each candidate value (plane-pass
 * variant 0/1/2, then the operand hints 0/1 (0-3 at n = 288), then the lookaheads 0 and 1/2, 1, 3/2,
 * 2 waves of resident blocks from the occupancy of this GPU, then the line form 0-4 at n = 288), keep
 * the fastest per key, each key timed with the
 * choices already made for the keys before it, and write the chosen values to chosen_host
 * [SGW_TUNE_KEYS] (may be NULL).  Needs sgw_set_potential and a spectral interval (SGW_ESTATE
 * otherwise); 1 <= batch <= max_batch and reps >= 1 (SGW_EINVAL otherwise).  Uses a context work
 * area of 2 batch-sized complex arrays (SGW_ENOMEM if it cannot grow).  Synchronises; must not be
 * called inside a stream capture.
 */
sgw_status sgw_autotune(sgw_ctx* ctx, int batch, int reps, int* chosen_host);

/*
 * Set H0 = T + V_loc + V_NL (Eq. 1 with the ionic pseudopotential split into a local
 * part, folded with V_H[rho0] + V_xc into vloc, and Kleinman-Bylander projectors).
 *  vloc_dev: [N_g] float, local potential (copied; the caller may free it afterwards).
 *  KB part (Sec. 3: atomic operations where neighbouring atoms' spheres overlap):
 *  n_atoms >= 0 atoms; atom a has nproj_host[a] in 1..4 projectors sharing the support
 *  sup_idx_host[sup_off_host[a] .. sup_off_host[a+1]) (flat grid indices, each < N_g,
 *  no repeats within an atom); beta_host holds, for each support point s of the whole
 *  list, 4 floats beta_ap(r_s) (unused p padded), i.e. [total_support][4];
 *  e_host is [n_atoms][4] projector energies E_ap.
 *  V_NL psi = sum_{a,p} beta_ap E_ap dV sum_r beta_ap(r) psi(r).
 * All host arrays are copied.  Passing n_atoms = 0 removes the nonlocal part.
 */
sgw_status sgw_set_potential(sgw_ctx* ctx, const float* vloc_dev, int n_atoms,
                             const int* nproj_host, const int64_t* sup_off_host,
                             const int* sup_idx_host, const float* beta_host,
                             const float* e_host);

/* out_dev = H0 in_dev for a batch of B c64 vectors (test hook and the building block of
 * every other call).  in and out may not alias. */
sgw_status sgw_apply_h(sgw_ctx* ctx, const void* in_dev, void* out_dev, int batch);

/*
 * Spectral bounds by shifted power iteration (Sec. 2.1): n_iter power steps on H0 give
 * E_max (Rayleigh quotient of the last iterate), n_iter steps on H0 - E_max give
 * E_min - E_max.  The start vector is the Philox white noise of (seed, stream 0xB0B0,
 * sample 0, vector 0).  The returned bounds are widened by margin * (E_max - E_min)
 * on each side; raw_host (optional, 2 doubles) receives the unwidened estimates.
 * The widened bounds are also stored in the context as the Chebyshev interval used by
 * the filter and the propagators.  Synchronises.
 */
sgw_status sgw_spectral_bounds(sgw_ctx* ctx, int n_iter, uint64_t seed, double margin,
                               double* emin_host, double* emax_host, double* raw_host);

/* Set the Chebyshev interval [emin, emax] directly (H~ = (H - Ebar)/dE maps it to [-1,1]). */
sgw_status sgw_set_spectrum(sgw_ctx* ctx, double emin, double emax);

/*
 * Coefficients a_0..a_{n_cheb} of the gapped Heaviside filter (Eq. 3), computed on the
 * host in FP64: the least-squares fit of the step function at the 4 (n_cheb + 1)
 * Chebyshev-Gauss nodes of [-1, 1], with zero weight for nodes inside
 * [x(E_HOMO), x(E_LUMO)], plus ridge * M * |a|^2 (M the node count), solved through the
 * normal equations: over all nodes the Gram matrix of T_0..T_N is diagonal (discrete
 * orthogonality), so removing the gap nodes is a low-rank correction solved with the
 * Woodbury identity and a Cholesky factorisation of the (gap nodes)^2 capacitance matrix.
 * x(E) = (E - Ebar)/dE for the interval [emin, emax].
 * coeffs_host: n_cheb + 1 doubles.  No context needed.
 */
sgw_status sgw_gapped_filter_coeffs(double e_homo, double e_lumo, double emin, double emax,
                                    int n_cheb, double ridge, double* coeffs_host);

/*
 * Chebyshev propagator coefficients for e^{-i H dt} on [emin, emax] (host, FP64, no context):
 * coeffs_host[2k], [2k+1] = re, im of (2 - delta_k0) (-i)^k J_k(dE |dt|), k = 0..cheb_deg
 * (complex conjugated for dt < 0), and phase_host[0..1] = e^{-i Ebar dt}.  J_k by Miller's
 * backward recurrence.  These are the coefficients sgw_propagate, sgw_tdh_response and
 * sgw_sigma_c use.
 */
sgw_status sgw_propagator_coeffs(double emin, double emax, double dt, int cheb_deg, double* coeffs_host,
                                 double* phase_host);

/*
 * Filtering (Eq. 3, Sec. 2.1): out = sum_{n=0}^{n_cheb} a_n T_n(H~) in, for a batch of c64
 * vectors, by the Clenshaw recurrence in FP32 on the context's interval.  in and out may
 * alias (in place).
 */
sgw_status sgw_filter_occupied(sgw_ctx* ctx, const double* coeffs_host, int n_cheb,
                               const void* in_dev, void* out_dev, int batch);

/*
 * Philox4x32-10 white noise (Sec. 2.1 white-noise start orbitals): out[s][v] for
 * s < n_samples, v < n_vec is the real Rademacher vector +-1/sqrt(dV) of
 * (seed, stream_id, sample = sample0 + s, vector = v), stored as c64 with zero
 * imaginary part.  Point g uses counter (g/4, v, sample, stream_id), key
 * (seed mod 2^32, seed div 2^32), output word g mod 4, sign from its top bit.
 */
sgw_status sgw_white_noise(sgw_ctx* ctx, uint64_t seed, uint32_t stream_id, int sample0,
                           int n_samples, int n_vec, void* out_dev);

/*
 * Split filtered white noise into the per-sample inputs of the two phases of Sec. 2.1.
 * noise_dev, filt_dev: [n_samples][n_eta + 1] c64, the white noise and its filtered image
 * (vector 0 of a sample is zeta-bar, vectors 1..n_eta the eta-bar_l).  Writes
 *  eta_dev [n_samples][n_eta] c64: eta_l = P eta-bar_l;
 *  zeta_dev [n_samples][2] c64: (zeta_occ = P zeta-bar, zeta_unocc = zeta-bar - P zeta-bar);
 *  source_dev [n_samples][N_g] float: Re(zeta-bar) * phi, the source of the TDH kick.
 * phi_dev: [N_g] float target orbital.
 */
sgw_status sgw_prepare_sample(sgw_ctx* ctx, const void* noise_dev, const void* filt_dev, const float* phi_dev,
                              int n_samples, int n_eta, void* eta_dev, void* zeta_dev, float* source_dev);

/*
 * Plain propagation under H0: psi <- (e^{-i H0 dt})^{n_steps} psi for a batch of c64
 * vectors (in place), each step the degree-cheb_deg Chebyshev expansion with Bessel
 * coefficients (2 - delta_k0) (-i)^k J_k(dE |dt|) and phase e^{-i Ebar dt}; dt < 0
 * propagates backwards.  dir_host (optional, [batch] int8: +1/-1) flips the direction
 * of individual vectors (NULL: all +1).
 */
sgw_status sgw_propagate(sgw_ctx* ctx, void* psi_dev, int batch, int n_steps, double dt,
                         int cheb_deg, const int8_t* dir_host);

/*
 * Plain propagation by the split-operator scheme (the paper's own time stepper, Sec. 3): each of
 * the n_steps steps applies, right to left,
 *   S(dt) = K_desc(dt/2) e^{-i V_loc dt/2} e^{-i T dt} e^{-i V_loc dt/2} K_asc(dt/2),
 * with e^{-i T dt} exact in k space (two xy-plane passes and one z-pencil pass) and the KB part
 * split atom by atom, e^{-i tau V_a} = 1 + Q_a (e^{-i tau M_a} - 1) Q_a^T (Q_a R_a = sqrt(dV) beta_a,
 * M_a = R_a E_a R_a^T), atoms grouped into colours of disjoint supports (greedy in atom order),
 * K_asc applying colours 0, 1, .. and K_desc the reverse.  Second order in dt, unitary to
 * rounding, time reversible.  psi_dev [batch][N_g] c64 in place; dir_host as in sgw_propagate.
 * SGW_ESTATE without a potential; SGW_EINVAL on a row-path grid (n = 48, 96, 288); graph mode as
 * in sgw_propagate.
 */
sgw_status sgw_propagate_split(sgw_ctx* ctx, void* psi_dev, int batch, int n_steps, double dt,
                               const int8_t* dir_host);

/*
 * Linear-response TDH (Sec. 2.1, first phase) for n_samples Monte-Carlo samples.
 *  eta_dev: [n_samples][n_eta] c64 filtered occupied stochastic orbitals (read only).
 *  source_dev: [n_samples][N_g] float, the source zeta-bar * phi of each sample.
 *  The perturbed copy of each eta is carried as its derivative with respect to the
 *  kick strength (tangent-linear pair, the lambda -> 0 limit of the perturbed-minus-
 *  unperturbed difference): d eta(0) = -i v_p eta(0), v_p = v_C * source.  Each step
 *  holds H(t_j) = H0 + v_C * (rho(t_j) - rho(0)), rho = weight * sum_l |eta_l|^2 fixed
 *  (weight <= 0 selects 2/n_eta).
 *  uR_dev: [n_samples][n_steps + 1][N_g] float receives u^R(t_j) = v_C * d rho(t_j).
 *  Requires 2 * n_samples * n_eta <= max_batch.
 *  cheb_deg >= 1: each step is the degree-cheb_deg Chebyshev expansion (needs a spectral
 *  interval); cheb_deg = 0: the split-operator step of sgw_propagate_split with V = V_loc +
 *  v_C * (rho(t_j) - rho(0)), its tangent taking the source -i (dt/2) d v psi in each local
 *  half-step (d v = v_C * d rho(t_j)).
 */
sgw_status sgw_tdh_response(sgw_ctx* ctx, const void* eta_dev, const float* source_dev,
                            int n_samples, int n_eta, int n_steps, double dt, int cheb_deg,
                            double weight, float* uR_dev);

/*
 * Time ordering: u(t_j), j = 0..n_steps, from the causal u^R(t_j) of each grid point
 * and sample: zero-pad to M (the smallest power of two >= 4 (n_steps + 1), M <= 4096),
 * FFT with e^{+i omega t}, replace the negative-frequency half by its complex conjugate,
 * inverse FFT.  uR_dev: [n_samples][n_steps+1][N_g] float; u_dev: same shape, c64.
 */
sgw_status sgw_time_order(sgw_ctx* ctx, const float* uR_dev, void* u_dev, int n_samples,
                          int n_steps);

/* The same time ordering for series of any length n_points per step ([n_samples][n_steps+1]
 * [n_points]): used for the xi-compressed U_m(t) of sgw_tdh_response_xi (n_points = n_xi). */
sgw_status sgw_time_order_points(sgw_ctx* ctx, const float* uR_dev, void* u_dev, int n_samples, int n_steps,
                                 int n_points);

/*
 * Sparse stochastic compression of u^R (Sec. 2.1 second paragraph, Sec. 2.3): instead of u^R on the
 * full grid, carry U_m(t_j) = <xi_m|u^R(t_j)>, m < n_xi, for random functions xi_m on fragmented
 * segments.  Reading of the construction: xi_m of MC sample (sample0 + s) is the sum of
 * K = max(1, round(N_g f_g / L)) draws, draw k covering the L (<= 32, dividing N_g) contiguous flat
 * grid points from L p with p = floor(w0 (N_g / L) / 2^32) and the sign of point l from bit l of w1
 * (set -> -1), (w0, w1) = Philox4x32-10 words of counter (k, m, sample, xi_stream) and key xi_seed,
 * times c = 1 / sqrt(n_xi K L dV / N_g), so that E[dV sum_m xi_m xi_m^T] = 1.
 *  sgw_tdh_response_xi: as sgw_tdh_response, but writes U_dev [n_samples][n_steps+1][n_xi] float
 *   (U_m(t_j) = dV sum_r xi_m(r) u^R(r, t_j)) instead of the full-grid u^R.  Time-order U with
 *   sgw_time_order_points(..., n_points = n_xi).
 *  sgw_sigma_c_xi: as sgw_sigma_c with u_dev [n_samples][n_steps+1][n_xi] c64 the time-ordered U:
 *   Sigma(+-t_j) = +-sum_m U_m(t_j) dV sum_r phi zeta(r, +-t_j) xi_m(r).
 * The same (xi_seed, xi_stream, sample0) must be passed to both.  SGW_EINVAL for n_xi < 1,
 * f_g <= 0, L outside 1..32 or not dividing N_g, sample0 < 0.
 */
sgw_status sgw_tdh_response_xi(sgw_ctx* ctx, const void* eta_dev, const float* source_dev, int n_samples, int n_eta,
                               int n_steps, double dt, int cheb_deg, double weight, uint64_t xi_seed,
                               uint32_t xi_stream, int sample0, int n_xi, double f_g, int L, float* U_dev);
sgw_status sgw_sigma_c_xi(sgw_ctx* ctx, void* zeta_dev, const float* phi_dev, const void* u_dev, int n_samples,
                          int n_steps, double dt, int cheb_deg, int fp64_accum, uint64_t xi_seed, uint32_t xi_stream,
                          int sample0, int n_xi, double f_g, int L, double* sigma_dev);

/*
 * zeta propagation and Sigma(t) (Eq. 4, Eq. 5): for each sample, zeta_unocc propagates
 * forward and zeta_occ backward under H0 for n_steps steps, and
 *   Sigma(+t_j) =  dV sum_r phi(r) zeta_unocc(r, t_j) u(r, t_j),
 *   Sigma(-t_j) = -dV sum_r phi(r) zeta_occ(r, -t_j) u(r, t_j),
 * with the two one-sided limits averaged at t = 0.
 *  zeta_dev: [n_samples][2] c64, (zeta_occ, zeta_unocc) per sample; propagated in place.
 *  phi_dev: [N_g] float target orbital; u_dev: [n_samples][n_steps+1][N_g] c64.
 *  sigma_dev: [n_samples][2 n_steps + 1] complex128 (index j + n_steps), written.
 *  fp64_accum = 1 accumulates the reductions in FP64, 0 in FP32.
 *  Requires 2 * n_samples <= max_batch.  cheb_deg = 0 propagates by the split-operator step of
 *  sgw_propagate_split instead of the degree-cheb_deg Chebyshev expansion.
 */
sgw_status sgw_sigma_c(sgw_ctx* ctx, void* zeta_dev, const float* phi_dev, const void* u_dev,
                       int n_samples, int n_steps, double dt, int cheb_deg, int fp64_accum,
                       double* sigma_dev);

/*
 * sROI exchange (Eq. 6): x_dev[s] = -(1/n_eta) sum_l <phi eta_l | v_C | phi eta_l> in FP64,
 * evaluated in k space.  eta_dev: [n_samples][n_eta] c64.  Requires n_eta <= max_batch.
 */
sgw_status sgw_exchange(sgw_ctx* ctx, const void* eta_dev, const float* phi_dev,
                        int n_samples, int n_eta, double* x_dev);

/*
 * Sigma(omega) (Eq. 7, trapezoid over t_j, end weights 1/2):
 *  out[w] = dt sum_j w_j Sigma(t_j) e^{-gamma^2 t_j^2/2} e^{i omega_w t_j}, j = -n_steps..n_steps,
 * for the mean over n_samples rows of sigma_dev.  omega_dev: [n_omega] double;
 * out_dev: [n_omega] complex128.  fp64 = 0 evaluates in FP32.
 */
sgw_status sgw_sigma_omega(sgw_ctx* ctx, const double* sigma_dev, int n_samples, int n_steps,
                           double dt, double gamma, const double* omega_dev, int n_omega,
                           int fp64, double* out_dev);

/*
 * QP equation (Eq. 6): the root of w = eps_ks + X + Re Sigma(w) - vxc nearest eps_ks for
 * the sample means of Sigma(t) (sigma_dev [n_samples][2 n_steps + 1] complex128) and X
 * (x_dev [n_samples] double): scan eps_ks +- window in steps of `step` for sign changes,
 * take the bracket nearest eps_ks, bisect to 1e-10 Ha.  The standard error is
 * Z * std_i(X_i + Re Sigma_i(eps_qp)) / sqrt(n_samples), Z = 1/(1 - dRe Sigma/dw).
 * result_host: [4] doubles = (eps_qp, standard error, Re Sigma(eps_qp), Z).
 * fp64 = 0 evaluates the transform in FP32.  Synchronises.  SGW_ENOCONV if no root.
 */
sgw_status sgw_qp_energy(sgw_ctx* ctx, const double* sigma_dev, const double* x_dev,
                         int n_samples, int n_steps, double dt, double gamma, double eps_ks,
                         double vxc, double window, double step, int fp64,
                         double* result_host);

/* ----------------------------------------------------------------------------------------
 * Learned control variate around the plain estimator of Sigma_c(t) (Eq. 4-5).  A sample's
 * Sigma_i(t) is a quadratic form in its random vector zeta-bar_i, so a network of cheap
 * features of zeta-bar_i predicts part of it; the paired estimator
 *   Sigma-hat = mean_{j<M} f(x_j) + mean_{i<n} (Y_i - f(x_i))
 * over M cheap samples (features only) and n full samples stays unbiased for any f.
 * ---------------------------------------------------------------------------------------- */

/* Number of features for shells 0 < |m|^2 <= m2max: 2 * (number of +-m pairs + 1). */
int sgw_cv_feature_count(int m2max);

/*
 * Features of n_samples Monte-Carlo samples from their white-noise vectors noise_dev
 * [n_samples][n_vec][N_g] c64 (vector 0 = zeta-bar, 1..n_vec-1 = eta-bar_l, as drawn by
 * sgw_white_noise).  For a vector v, F_v(k) = dV sum_r Re v(r) phi(r) e^{-i k.r} at k = 2 pi m / L
 * for 0 < |m|^2 <= m2max (one of each +-m pair: first non-zero component of m positive;
 * ordered by |m|^2, then (mx, my, mz) lexicographically), weighted by sqrt(4 pi)/|k|.
 * feat_dev[s] (float, sgw_cv_feature_count(m2max) entries) = [|F_zeta(k)|^2 for each k,
 * F_zeta(0)^2, sum_l |F_eta_l(k)|^2 for each k, sum_l F_eta_l(0)^2].  Requires n_vec <= max_batch.
 */
sgw_status sgw_cv_features(sgw_ctx* ctx, const void* noise_dev, int n_samples, int n_vec, const float* phi_dev,
                           int m2max, float* feat_dev);

/* Column means and sample standard deviations (FP64; 1 where zero) of y_dev [n_rows][n_out]
 * (double) into mu_dev, sd_dev when compute_stats != 0, and t_dev = (y - mu) / sd as float. */
sgw_status sgw_cv_standardize(sgw_ctx* ctx, const double* y_dev, int n_rows, int n_out, int compute_stats,
                              double* mu_dev, double* sd_dev, float* t_dev);

/* The same for float columns, in place: x = (x - mu) / sd. */
sgw_status sgw_cv_standardize_f32(sgw_ctx* ctx, float* x_dev, int n_rows, int n_cols, int compute_stats,
                                  double* mu_dev, double* sd_dev);

/*
 * Control-variate rows (FP64): rows_dev[i][o] = mean_j f_j[o] + y_i[o] - f_i[o] with
 * f = mu + sd * (network output), f_cheap_dev [n_cheap][n_out] and f_paired_dev [n_paired][n_out]
 * the network outputs (float) of the cheap and of the paired samples, y_paired_dev the paired
 * samples' targets (double).  The mean of the rows is the control-variate estimate and their
 * spread its sample standard deviation, so they can be passed to sgw_qp_energy as the samples of
 * Sigma(t) (viewing each complex128 Sigma row as 2 (2 N + 1) doubles).  n_cheap = 0 means f = 0:
 * the rows are then exactly y (the plain estimator).
 */
sgw_status sgw_cv_rows(sgw_ctx* ctx, const float* f_cheap_dev, int n_cheap, const float* f_paired_dev,
                       const double* y_paired_dev, int n_paired, int n_out, const double* mu_dev,
                       const double* sd_dev, double* rows_dev);

/*
 * Linear part of the control variate (not in the paper).  The per-k features of sgw_cv_features
 * are summed per shell |m|^2 (the distinct |m|^2 <= m2max, increasing): out_dev[i] =
 * [zeta-bar shell sums..., zeta-bar k = 0 feature, eta-bar shell sums..., eta-bar k = 0 feature]
 * (float, sgw_cv_shell_count(m2max) = 2 (shells + 1) per sample; sums accumulated in FP64 in the
 * features' k order).  feat_dev [n_samples][sgw_cv_feature_count(m2max)] (float).
 */
int sgw_cv_shell_count(int m2max);
sgw_status sgw_cv_shell_sums(sgw_ctx* ctx, const float* feat_dev, int n_samples, int m2max, float* out_dev);

/*
 * FP64 ridge regression of targets y_dev [n][o] (double) on inputs x_dev [n][p] (float):
 * mu, sd = column means and sample standard deviations of x (1 where 0), Xs = (x - mu) / sd,
 * ybar = column means of y, and B solves (Xs^T Xs + ridge n I) B = Xs^T (y - ybar) (Gram and cross
 * products on the GPU in FP64, Cholesky on the host in FP64).  model_dev (double, caller-owned,
 * sgw_cv_linear_size(p, o) = 2p + o + p o entries) receives [mu][sd][ybar][B (p x o, row-major)].
 * Needs n >= 2, 1 <= p <= 256, o >= 1, ridge >= 0 (SGW_EINVAL otherwise); SGW_ENOCONV when the
 * normal matrix is not positive definite (ridge = 0 with dependent columns).  Synchronises.
 */
int64_t sgw_cv_linear_size(int p, int o);
sgw_status sgw_cv_linear_fit(sgw_ctx* ctx, const float* x_dev, const double* y_dev, int n, int p, int o, double ridge,
                             double* model_dev);

/* f_ij = ybar_j + sum_a ((x_ia - mu_a) / sd_a) B_aj  (FP64) for x_dev [n][p] (float); out_dev [n][o]
 * receives f, or y_dev - f (the residual of targets y_dev [n][o]) when y_dev is not NULL. */
sgw_status sgw_cv_linear_apply(sgw_ctx* ctx, const double* model_dev, const float* x_dev, int n, int p, int o,
                               const double* y_dev, double* out_dev);

/*
 * Rows of the linear control variate (FP64): y_out_dev[i][j] = y_i[j] - f(x_i)[j] + mean_m f(xc_m)[j]
 * for the paired samples' inputs x_paired_dev [n_paired][p] and targets y_dev [n_paired][o] and
 * the cheap samples' inputs x_cheap_dev [n_cheap][p] (the mean of a linear f is f at the mean
 * input).  The rows' mean is unbiased for E[y] whatever the model; they can be combined further
 * with sgw_cv_rows (network part) or passed to sgw_qp_energy.  n_cheap, n_paired >= 1.
 */
sgw_status sgw_cv_linear_rows(sgw_ctx* ctx, const double* model_dev, const float* x_cheap_dev, int n_cheap,
                              const float* x_paired_dev, int n_paired, int p, int o, const double* y_dev,
                              double* y_out_dev);

/*
 * The network: h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), h3 = tanh(h2 W3 + b3),
 * y = h3 W4 + b4, with n_in inputs, three hidden layers of `width`, n_out outputs.  FP32 master
 * weights and Adam state; the matrix products run on the tensor cores with BF16 operands
 * (weights, activations, back-propagated errors) and FP32 accumulation.  Loss: mean over the
 * batch and outputs of (y - t)^2.  Parameters are ordered W1, b1, W2, b2, W3, b3, W4, b4, each
 * matrix row-major [in][out].  Initial weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from
 * splitmix64(seed), biases 0.  max_batch bounds M in every call.
 */
typedef struct sgw_mlp sgw_mlp;
sgw_status sgw_mlp_create(sgw_mlp** out, int n_in, int width, int n_out, int max_batch, uint64_t seed,
                          int device, void* stream);
void sgw_mlp_destroy(sgw_mlp* m);
const char* sgw_mlp_last_error(const sgw_mlp* m);
int64_t sgw_mlp_param_count(const sgw_mlp* m);
/* Replace the parameters (host float array of sgw_mlp_param_count entries); resets Adam. */
sgw_status sgw_mlp_set_params(sgw_mlp* m, const float* params_host, int64_t n);
sgw_status sgw_mlp_get_params(sgw_mlp* m, float* params_host, int64_t n);
/* Per-output loss weights w_o (loss = sum_o w_o (y - t)^2 / (M n_out)); NULL restores 1. */
sgw_status sgw_mlp_set_loss_weights(sgw_mlp* m, const float* w_host, int n_out);
/* y_dev [M][n_out] = network(x_dev [M][n_in]) (float). */
sgw_status sgw_mlp_forward(sgw_mlp* m, const float* x_dev, int M, float* y_dev);
/* Loss and gradients for a batch (kept for sgw_mlp_adam_step); loss_host and grads_host
 * (sgw_mlp_param_count floats) are optional and synchronise when given. */
sgw_status sgw_mlp_gradients(sgw_mlp* m, const float* x_dev, const float* t_dev, int M, double* loss_host,
                             float* grads_host);
/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8) with the last gradients. */
sgw_status sgw_mlp_adam_step(sgw_mlp* m, float lr);
/* One pass over n_rows rows in consecutive mini-batches of `batch` (gradients + Adam each). */
sgw_status sgw_mlp_train_epoch(sgw_mlp* m, const float* x_dev, const float* t_dev, int n_rows, int batch,
                               float lr, double* mean_loss_host);

/*
 * QP solve that allocates nothing (no counterpart in the paper).  For callers that cannot let
 * a library allocate device memory -- e.g. a host application that has reserved the device's
 * memory for its own pool allocator, or a plugin host that forbids allocations while it runs.
 * Same computation and arguments as sgw_qp_energy, without a context: sigma_dev, x_dev and the
 * work run on `stream` (a cudaStream_t, NULL = default) on the current device.  Scratch is a
 * fixed 1 MiB device array inside the library (held on every GPU that loads the library until
 * exit).  With n_scan = round(2 window/step) + 1 scan points, a call needs
 * (n_scan rounded up to even) + 2 (2 n_steps + 1) + 4 doubles; calls that need more than 131072
 * doubles, or whose 2 window/step is not finite, are rejected with SGW_EINVAL.  Outside a stream
 * capture every call looks up the array's device address on the current device (so the call
 * also works after the application resets and re-creates the device's context); during a capture
 * the address found by an earlier call on that device is used, so make the first call on a
 * device before any stream capture (otherwise SGW_ESTATE).  All calls on a device share the
 * array and nothing in it is kept between calls: calls that overlap on the GPU (other streams or
 * threads) race and must be serialised by the caller.  Errors are reported through
 * sgw_last_error(NULL).  Synchronises `stream`.
 */
sgw_status sgw_qp_energy_noalloc(const double* sigma_dev, const double* x_dev, int n_samples,
                                 int n_steps, double dt, double gamma, double eps_ks, double vxc,
                                 double window, double step, int fp64, double* result_host,
                                 void* stream);

/*
 * Instrumentation (no counterpart in the paper beyond its per-portion wall times, Table 4).
 * Kernel kinds for sgw_profile_read:                                                      */
enum {
    SGW_PROF_PLANE_STEP = 0,   /* fused xy-plane pass of a Chebyshev term (inverse FFT, V psi,
                                  KB apply, recurrence, forward FFT)                       */
    SGW_PROF_PENCIL = 1,       /* z-pencil pass (FFT along z, kinetic multiply, inverse)   */
    SGW_PROF_KB = 2,           /* KB projector contraction                                 */
    SGW_PROF_PLANE_FWD = 3,    /* forward xy-plane pass                                    */
    SGW_PROF_TDH_DENSITY = 4,  /* TDH density + forward xy pass of the Poisson solve       */
    SGW_PROF_SIGMA = 5,        /* Sigma(t) reduction                                       */
    SGW_PROF_TIME_ORDER = 6,   /* time ordering                                            */
    SGW_PROF_OTHER = 7,        /* everything else                                          */
    SGW_PROF_SPLIT_INV = 8,    /* inverse plane pass of a split-operator step              */
    SGW_PROF_LINES = 9,        /* y-line passes of the 288 grid's row form (16 bytes per
                                  vector-point each); the 36-row step is SGW_PROF_PLANE_STEP  */
    SGW_PROF_KINDS = 10
};

/* enable != 0: from now on record CUDA events on the context's stream around every kernel
 * launch; resets the accumulated times.  Synchronises. */
sgw_status sgw_profile(sgw_ctx* ctx, int enable);

/* Accumulated device time (ms, from the recorded events), launch count and algorithmic
 * (compulsory) HBM bytes of one kernel kind since sgw_profile(ctx, 1): for a plane pass
 * 8 bytes per vector-point for each complex array it must read or write, 4 per point for
 * each potential row; for a pencil pass 16 per vector-point; for the KB contraction 8 per
 * support point and vector plus the projector table.  alg_bytes_host may be NULL.
 * Synchronises. */
sgw_status sgw_profile_read(sgw_ctx* ctx, int kind, double* total_ms_host, int64_t* count_host,
                            double* alg_bytes_host);

/* Number of kernels this context has launched since it was created. */
sgw_status sgw_launch_count(sgw_ctx* ctx, int64_t* count_host);

#ifdef __cplusplus
}
#endif

#endif /* SGW_H */
