// Internal declarations shared by the translation units of libsgw.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgw {

// Per-vector description for the fused Chebyshev step.
struct VecInfo {
    int vrow;     // row of the local potential table used by this vector
    int dvrow;    // row of the tangent potential (-1: not a tangent vector)
    int partner;  // batch index of the vector whose b_{k+1} couples through dvrow
    int cset;     // coefficient set (0 forward / 1 backward)
};

// Coefficients of one fused step, per coefficient set:
//   out = cpsi * psi + ch * alpha * (H b1 - ebar b1 [+ dv * b1_partner]) + c2 * b2
struct StepCoef {
    float2 cpsi[2];
    float2 ch[2];
    float2 c2[2];
};

struct KBDev {
    int n_atoms = 0;
    int n_proj = 0;            // 4 * n_atoms (padded)
    int64_t n_sup = 0;
    int* atom_nproj = nullptr;   // [n_atoms]
    int64_t* atom_off = nullptr; // [n_atoms + 1]
    int* sup_idx = nullptr;      // [n_sup]
    float4* sup_beta = nullptr;  // [n_sup]   beta_a0..3 at each support point
    float4* atom_e = nullptr;    // [n_atoms] E_a0..3
    // per-unit partial projections (a unit is an xy plane on the plane path, 8 x rows on the row
    // path): unit z owns slots plane_off[z] .. plane_off[z+1]-1, one per atom whose support meets
    // the unit (slot_atom[k] is that atom); atom a's slots (in increasing z) are
    // atom_pos[atom_pos_off[a] .. atom_pos_off[a+1]).
    int total_slots = 0;
    int max_plane_slots = 0;
    int* plane_off = nullptr;    // [units + 1]
    int* slot_atom = nullptr;    // [total_slots]
    // plane-major entries of the fused apply and projections.  The slots of a plane are split into
    // colours whose point sets in the plane are disjoint; plane z's colour c holds the entries
    // kbe_col[z (max_colors+1) + c] .. kbe_col[z (max_colors+1) + c + 1] - 1, slot by slot
    // (slot k: kbe_slot_beg[k] .. kbe_slot_end[k] - 1).  Entry e: kbe_os[e] = in-plane offset |
    // (plane-local slot << 16), kbe_beta[e] = the slot atom's beta_0..3 at that point.
    int max_colors = 0;
    int* kbe_col = nullptr;      // [units][max_colors + 1]
    unsigned* kbe_os = nullptr;  // [n_sup]
    float4* kbe_beta = nullptr;  // [n_sup]
    int* kbe_slot_beg = nullptr; // [total_slots]
    int* kbe_slot_end = nullptr; // [total_slots]
    int* atom_pos_off = nullptr; // [n_atoms + 1]
    int* atom_pos = nullptr;     // [total_slots]
};

struct StepArgs {
    const float2* W;        // [B][ng] input planes in the xy-transformed / z-filtered representation
                            // (the row path transforms it back along y in place: W is dead afterwards)
    float2* Wout;           // [B][ng] forward xy transform of the output (nullptr: skip)
    const float2* b1;       // [B][ng] real-space vector H acts on
    const float2* b2;       // [B][ng] real-space b_{k+2} (nullptr when c2 == 0)
    const float2* psi;      // [B][ng] real-space psi (nullptr when cpsi == 0)
    float2* out;            // [B][ng] real-space output
    const float* vpot;      // [rows][ng]
    const float* dvpot;     // [rows][ng] or nullptr
    const VecInfo* info;    // [B]
    const float2* kbc;      // [B][n_proj] E-weighted projector coefficients (nullptr: no KB)
    // KB tables (see KBDev)
    const int* plane_off;
    const int* slot_atom;
    const int* kbe_col;
    const unsigned* kbe_os;
    const float4* kbe_beta;
    const int* kbe_slot_beg;
    const int* kbe_slot_end;
    int max_colors;
    int max_plane_slots;
    // partial projections of `out` (nullptr: skip): kbp[b][slot][4] = sum_plane beta_ap(r) out(r)
    float2* kbp;
    int total_slots;
    int n_proj;
    float ebar, alpha;
    StepCoef coef;
    // L2 prefetch of the W plane of the block this many blocks later in launch order (0: off);
    // a performance hint only, results do not depend on it
    int pf_ahead;
    // 1: prefetch this block's pointwise operands into L2 at its start (a hint as well)
    int pf_operands;
};

// ---- grid kernels (kernels_grid.cu)
bool grid_supported(int n);
cudaError_t grid_init_attributes(int n);
int plane_step_blocks_per_sm(int n, int variant, int max_plane_slots);
size_t plane_step_smem(int n, int max_plane_slots);
size_t plane_pipe_smem(int n, int max_plane_slots);
bool plane_pipe_supported(int n);
cudaError_t plane_step_reserve_smem(int n, int max_plane_slots);
int pencil_blocks_per_sm(int n);
void launch_plane_fwd(int n, const float2* in, float2* W, int batch, const float2* tw, cudaStream_t st);
// kind: 0 kinetic (T(k)/N^3, capped at ecut if ecut > 0), 1 Coulomb (4 pi/k^2 / N^3, k=0 -> 0)
// line_form: form of the z-line pass on the 288 grid (0, 1, 2; a launch hint)
void launch_pencil(int n, float2* W, int batch, int kind, float kscale, float ecut, const float2* tw,
                   cudaStream_t st, int pf_ahead = 0, const VecInfo* info = nullptr, float dt = 0.f,
                   int line_form = 0);
void launch_plane_fwd_phase(int n, const float2* psi, const float* vpot, const float* dvpot, const VecInfo* info,
                            float dt, float2* W, int batch, const float2* tw, cudaStream_t st);
void launch_split_tangent(float2* psi, const float* dvpot, const VecInfo* info, float dt, int batch, int64_t ng,
                          cudaStream_t st);
void launch_plane_inv_phase(int n, const float2* W, const float* vloc, const VecInfo* info, float dt, float2* psi,
                            int batch, const float2* tw, cudaStream_t st);
void launch_kb_split(const int* atoms, int n_atoms_colour, const KBDev& kb, const float4* q4, const float2* F,
                     const VecInfo* info, float2* x, int batch, size_t ng, cudaStream_t st);
// exchange energy: acc[b / per] += (dV / N) sum_k v(k) |F(k)|^2 after the z transform
int pencil_blocks(int n);
void launch_pencil_coulomb_energy(int n, const float2* W, int batch, int per, float kscale, double dvn,
                                  const float2* tw, double* part, double* acc, cudaStream_t st);
void launch_plane_step(int n, const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int variant = 0,
                       int line_form = 0);
// inverse xy transform of W (in place along y on the row path; W is scratch), epilogue:
// mode 0 -> out_c[b] = plane (c64);
// mode 1 (Poisson of TDH densities) -> vtot[b] = vloc + Re, dv[b] = Im, uR[b] = Im (if uR)
void launch_plane_inv(int n, const float2* W, int batch, const float2* tw, int mode, float2* out_c,
                      const float* vloc, float* vtot, float* dv, float* uR, int64_t uR_stride,
                      float* out_re, cudaStream_t st);
void launch_kb_project(int n, const KBDev& kb, const float2* b1, int batch, float dV, float2* kbc,
                       cudaStream_t st);
// kbc[b][4a + p] = E_ap dV sum over atom a's plane slots of kbp[b][slot][p]
void launch_kb_reduce(const KBDev& kb, const float2* kbp, int batch, float dV, float2* kbc, cudaStream_t st);
// density of TDH pairs for each sample, packed as (rho - rho0) + i d rho, fwd xy transformed into Wp.
void launch_density_fwd(int n, const float2* psi, int n_samples, int n_eta, float weight, float* rho0,
                        int store_rho0, float2* Wp, const float2* tw, cudaStream_t st);

// ---- row path (kernels_rows.cu): grids of side 2^a 3^b (48, 96, 288) whose planes are split into
// units of 8 x rows; the launchers above dispatch to it for those sizes.  KB tables, slots and
// colours are per unit (unit_points(n) consecutive points: n^2 on the plane path, 8 n here).
bool rows_path(int n);
int64_t unit_points(int n);
int rows_units(int n);
size_t rows_step_smem(int n, int max_unit_slots);
cudaError_t rows_init_attributes(int n);
cudaError_t rows_step_reserve_smem(int n, int max_unit_slots);
int rows_step_blocks_per_sm(int n, int variant, int max_unit_slots);
int zlines_blocks_per_sm(int n);
void rows_plane_fwd(int n, const float2* in, float2* W, int batch, const float2* tw, cudaStream_t st);
void rows_pencil(int n, float2* W, int batch, int kind, float kscale, float ecut, const float2* tw, cudaStream_t st,
                 int line_form);
void rows_zlines_energy(int n, const float2* W, int batch, float kscale, const float2* tw, double* part,
                        cudaStream_t st);
void rows_plane_step(int n, const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int variant,
                     int line_form = 0);
void rows_plane_inv(int n, const float2* W, int batch, const float2* tw, int mode, float2* out_c, const float* vloc,
                    float* vtot, float* dv, float* uR, int64_t uR_stride, float* out_re, cudaStream_t st);
void rows_density_fwd(int n, const float2* psi, int n_samples, int n_eta, float weight, float* rho0, int store_rho0,
                      float2* Wp, const float2* tw, cudaStream_t st);

// ---- the 288 grid (kernels_cluster.cu): one thread-block cluster of 8 CTAs per xy plane for the
// fused step (units of 36 rows), z lines in one of three forms
bool cluster_plane(int n);
int cluster_unit_rows();
size_t cplane_smem(int max_unit_slots);
cudaError_t cluster_init_attributes(int max_unit_slots);
int cplane_blocks_per_sm(int variant, int max_unit_slots);
int zlines_reg_blocks_per_sm(int form);
// variant 0: the row form (y lines, 36-row step, y lines); 1, 2: one cluster of 8 CTAs per plane
// with 32 / 18 warps per CTA
// (line_form 3: the row form's y lines by the two-stage 16 x 18 transform; 4: its rows as well)
void cplane_step(const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int variant, int line_form = 0);
// form 0 / 1: register-ended Stockham tiles of 16 / 32 columns, 2: warp-FFT tiles of 16 columns,
// 3, 4: the two-stage 16 x 18 transform on tiles of 16 columns
void zlines_reg(float2* W, int batch, int kind, int form, float kscale, float ecut, const float2* tw, cudaStream_t st);
// the row form's passes one by one (the library times them separately): y lines in place on W
// (dir +1 inverse, -1 forward; forms 3, 4 two-stage, else radix stages) and the 36-row step (form
// 4: rows by the two-stage transform, else by warp FFTs)
void lines288(float2* W, int batch, int dir, int form, const float2* tw, cudaStream_t st);
void rows36_step(const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int form = 0);
// the two-stage 16 x 18 line transforms of the 288 grid (kernels_lines288.cu)
cudaError_t lines288_2s_init_attributes();
int lines288_2s_blocks_per_sm();
void ylines288_2s(float2* W, int batch, int dir, const float2* tw, cudaStream_t st);
void zlines288_2s(float2* W, int batch, int kind, float kscale, float ecut, const float2* tw, cudaStream_t st);
cudaError_t rows36_2s_init_attributes(int max_unit_slots);
int rows36_2s_blocks_per_sm(int max_unit_slots);
void rows36_2s_step(const StepArgs& a, int batch, const float2* tw, cudaStream_t st);

// ---- other kernels (kernels_misc.cu)
void launch_noise(int ng, uint64_t seed, uint32_t stream_id, int sample0, int n_samples, int n_vec,
                  float amp, float2* out, cudaStream_t st);
void launch_real_to_c64(int64_t count, const float* in, float2* out, cudaStream_t st);
void launch_kick(int ng, const float2* eta, const float* vp, int n_samples, int n_eta, float2* psi,
                 cudaStream_t st);
void launch_scale_mul(int64_t count, const float* phi, int ng, const float2* eta, float2* out, cudaStream_t st);
// power-iteration helpers (single vector, FP64 reductions into scal[])
void launch_dot2(int ng, const float2* v, const float2* w, double* scal, cudaStream_t st);
void launch_power_update(int ng, const float2* w, float2* v, const double* scal, double* est_out,
                         const double* shift, float dV, cudaStream_t st);
void launch_sigma_accum(int ng, const float2* zeta, const float* phi, const float2* u, int n_samples,
                        int64_t u_sample_stride, int j, int n_steps, float dV, int fp64, double2* partial,
                        int nblk, cudaStream_t st);
void launch_xi_project(const float* f, int64_t f_ss, int n_samples, int n_xi, int K, int L, int64_t ng, uint64_t seed,
                       uint32_t stream, int sample0, float cdv, float* U, int64_t u_ss, cudaStream_t st);
void launch_sigma_accum_xi(const float2* zeta, const float* phi, const float2* Uxi, int n_samples, int64_t u_ss, int j,
                           int n_steps, int n_xi, int K, int L, int64_t ng, uint64_t seed, uint32_t stream, int sample0,
                           float c, int fp64, double2* partial, int nblk, cudaStream_t st);
void launch_sigma_reduce(const double2* partial, int n_samples, int n_steps, int nblk, double dV, int fp64,
                         double* sigma, cudaStream_t st);
void launch_time_order(int ng, const float* uR, float2* u, int n_samples, int n_steps, int M,
                       const float2* twM, cudaStream_t st);
void launch_sigma_omega(const double* sigma, int n_samples, int n_steps, double dt, double gamma,
                        const double* omega, int n_omega, int fp64, double* out, cudaStream_t st);
void launch_qp(const double* sigma, const double* x, int n_samples, int n_steps, double dt, double gamma,
               double eps_ks, double vxc, double window, double step, int fp64, double* scan,
               int n_scan, double* result, cudaStream_t st);
int time_order_threads(int M);
void set_global_error(const char* msg);
// control variate (kernels_mlp.cu)
void launch_cv_source(int64_t ng, const float2* zb, int64_t stride, const float* phi, int n_samples, float2* out,
                      cudaStream_t st);
void launch_cv_gather(int n, const float2* W, int n_samples, int nk, const int4* ks, float kscale, float dV,
                      const float2* tw, float* feat, cudaStream_t st);
void launch_cv_stats(int n, int O, const double* y, double* mu, double* sd, cudaStream_t st);
void launch_cv_combine(int n_samples, int nv, int nk, const float* raw, float* feat, cudaStream_t st);
void launch_cv_standardize_f32(int n, int O, float* y, double* mu, double* sd, int compute, cudaStream_t st);
void launch_cv_standardize(int64_t total, int O, const double* y, const double* mu, const double* sd, float* t,
                           cudaStream_t st);
void launch_cv_shells(int n, int nk, int n_shells, const int* shell_of_k, const float* feat, float* out, cudaStream_t st);
void launch_f32_to_f64(int64_t n, const float* a, double* b, cudaStream_t st);
void launch_cv_gram(int n, int p, const double* x, const double* mu, const double* sd, double* G, cudaStream_t st);
void launch_cv_xty(int n, int p, int o, const double* x, const double* mu, const double* sd, const double* y,
                   const double* ybar, double* C, cudaStream_t st);
void launch_cv_lin_apply(int n, int p, int o, const double* m, const float* x, const double* y, double* out,
                         cudaStream_t st);
void launch_cv_lin_rows(int mc, int n, int p, int o, const double* m, const float* xc, const float* xp,
                        const double* y, double* xbar, double* yout, cudaStream_t st);
void launch_cv_rows(int Mc, int n, int O, const float* fc, const float* fp, const double* y, const double* mu,
                    const double* sd, double* rows, cudaStream_t st);
void launch_prepare(int ng, const float2* noise, const float2* filt, const float* phi, int n_samples, int n_eta,
                    float2* eta, float2* zeta, float* source, cudaStream_t st);

}  // namespace sgw
