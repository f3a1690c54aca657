/*
 * fde.h -- C ABI of the GB300 periodic frozen-density-embedding (subsystem DFT) library.
 *
 * The library computes the data-parallel hot path of periodic subsystem DFT
 * (Genova, Ceresoli & Pavanello, "Periodic Subsystem Density-Functional Theory",
 * arXiv:1406.7803): the embedded plane-wave Kohn-Sham apply H_I psi for every subsystem I,
 * the embedding-potential build that feeds it, the subsystem eigensolver and the
 * freeze-and-thaw cycle around them.  Everything on that path runs in the library's own
 * CUDA kernels on one GPU.
 *
 * Units: Hartree atomic units (bohr, Hartree).
 *
 * Conventions shared by every call:
 *   - grid functions are real arrays in C order [n1][n2][n3] (n3 fastest); grid point
 *     (i1,i2,i3) sits at sum_j (i_j/n_j) a_j.
 *   - orbitals u_jk(r) = Omega^{-1/2} sum_G c_G e^{iG.r}, sum_G |c_G|^2 = 1; a block of
 *     orbitals is band-major [nb][npw] of interleaved complex (re, im).  The sphere of one
 *     k-point holds every G with |k+G|^2/2 <= ecut (FP64 test on the integer Miller
 *     indices) sorted lexicographically by signed (m1, m2, m3) (fde_get_basis).
 *   - forward transform f(G) = (1/N_r) sum_r f(r) e^{-iG.r}; Nyquist planes (m_j = -n_j/2,
 *     n_j even) are zeroed in every reciprocal-space filter (Poisson, local potential,
 *     gradient, divergence).
 *
 * Memory: pointers named d_* are device pointers owned by the caller (the library never
 * frees or keeps them); pointers named h_* are host pointers owned by the caller.  The
 * library owns its context memory (allocated with cudaMalloc at fde_create /
 * fde_add_subsystem / first use, released by fde_destroy).  All device work is enqueued on
 * the stream given to fde_create; calls that return host values synchronise that stream.
 *
 * Errors: no exception crosses the ABI.  Every call returns an fde_status; on failure the
 * context keeps a message readable with fde_last_error.  A device-side status word is
 * checked at the end of each synchronising call and maps to FDE_ENONFINITE.
 */
#ifndef FDE_H
#define FDE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fde_ctx fde_ctx;

typedef enum {
  FDE_OK = 0,
  FDE_EINVAL = -1,        /* bad argument (null pointer, index out of range, bad size) */
  FDE_ENOMEM = -2,        /* device or host allocation failed */
  FDE_ECUDA = -3,         /* a CUDA runtime call failed */
  FDE_ENOCONV = -4,       /* an iteration reached its cap before its tolerance */
  FDE_ENONFINITE = -5,    /* a density, potential or energy became NaN/Inf */
  FDE_ETIMEOUT = -6,      /* a bounded device wait ran out (tensor-core products) */
  FDE_EUNSUPPORTED = -7   /* a size or option outside what the kernels handle */
} fde_status;

typedef enum {
  FDE_PREC_FP64 = 0,  /* everything in FP64 */
  FDE_PREC_MIXED = 1  /* FP32 orbitals, H psi transforms, subspace products and pointwise
                         functionals; double-float density and gradient transforms; FP64
                         dense algebra, densities, potentials in memory and energies; a
                         freeze-and-thaw cycle ends with an FP64 refinement */
} fde_prec;

enum { FDE_XC_LDA = 0, FDE_XC_PBE = 1 };                         /* exchange-correlation */
enum { FDE_KEDF_TF = 0, FDE_KEDF_REVAPBEK = 1, FDE_KEDF_LC94 = 2 };  /* kinetic functional */
enum { FDE_PRECOND_TPA = 0, FDE_PRECOND_LEARNED = 1 };          /* eigensolver preconditioner */
enum { FDE_SMEAR_FERMI = 0, FDE_SMEAR_MP = 1, FDE_SMEAR_GAUSS = 2 }; /* occupation smearing */
enum { FDE_PRECOND_PARAMS = 8641 };  /* learned-preconditioner parameter count (floats) */

/* Cell, shared real-space grid and wavefunction cutoff (Sec. 2: one shared grid holds rho
 * and every potential, Eq. meth:1).  lattice rows are a_1, a_2, a_3 (bohr); the cell must
 * be orthorhombic (diagonal lattice) -- other cells return FDE_EUNSUPPORTED.  Each grid
 * size must factor into 2, 3 and 5 and be at most 512. */
typedef struct {
  double lattice[3][3];
  int grid[3];
  double ecut_ha;
} fde_cell_desc;

/* Functionals (Computational Details: PBE xc with LC94 or revAPBEK nonadditive kinetic
 * energy; LDA and Thomas-Fermi are the simpler members of the same families). rho_cut:
 * points with rho < rho_cut contribute no energy density and no potential. */
typedef struct {
  int xc;
  int kedf;
  double rho_cut;
} fde_func_desc;

/* One subsystem (Sec. 2: subsystem density with BZ integral and fractional occupations;
 * Appendix: subsystem-specific projectors).  pos [natoms][3] bohr, Z [natoms]; every atom
 * carries the local potential -Z erf(|r-R|/rc)/|r-R| and nproj_per_atom Gaussian s-type
 * Kleinman-Bylander projectors of widths proj_sigma [nproj_per_atom] (bohr) coupled by
 * proj_D [nproj_per_atom][nproj_per_atom] (Ha, symmetric; nproj_per_atom <= 8, else
 * FDE_EUNSUPPORTED).  kpts [nk][3] in crystal
 * coordinates with weights wk [nk] summing to 1 (a full Monkhorst-Pack mesh or its
 * irreducible part from fde_host_kmesh).  smearing_ha > 0: smeared occupations of kind
 * smearing_kind (Computational Details: Methfessel-Paxton for the metallic subsystems;
 * FDE_SMEAR_MP is the first-order form, FDE_SMEAR_GAUSS the zeroth, FDE_SMEAR_FERMI
 * Fermi-Dirac); 0: integer occupations (then nk must be 1 and nelec/2 an integer <= nbands).
 * aug_sigma > 0 makes the atoms ultrasoft-like (Appendix: PAW / ultrasoft pseudopotentials with
 * subsystem-specific projectors; here a model of them): the projectors also define the overlap
 * S_I = 1 + sum_{a in I} sum_ij |beta_ai> q_ij <beta_aj| with proj_Q = q [nproj_per_atom]^2
 * (symmetric, positive definite), the subsystem's eigenproblem becomes H_I psi = e S_I psi, its
 * density gains the augmentation charges q_ij g_a(r) <psi|beta_ai><beta_aj|psi> with g_a the
 * normalised Gaussian (pi aug_sigma^2)^{-3/2} exp(-|r - R_a|^2 / aug_sigma^2), and each atom's
 * coupling is screened, D_a = D + q int V_eff^I g_a.  aug_sigma = 0: norm-conserving (proj_Q
 * unused).  All arrays are host memory and are copied. */
typedef struct {
  int natoms;
  const double* pos;
  const double* Z;
  double rc;
  int nproj_per_atom;
  const double* proj_sigma;
  const double* proj_D;
  int nbands;
  int nk;
  const double* kpts;
  const double* wk;
  double nelec;
  double smearing_ha;
  int smearing_kind;
  const double* proj_Q;
  double aug_sigma;
} fde_subsys_desc;

/* Energy terms of Eq. E_FDE (Sec. 2) for the current densities and orbitals:
 *   E_fde = E_kin + E_nl + E_loc + E_H + E_xc + T_nad + E_nn
 * with E_kin = sum_I T_J[rho_I] (Janak), E_nl the subsystem-specific nonlocal energy,
 * E_loc = int v_loc rho (all nuclei), E_H = E_H[rho], E_xc = E_xc[rho],
 * T_nad = T~[rho] - sum_I T~[rho_I], E_nn the Ewald nuclear repulsion.  TS = sum_I sigma_I S_I
 * (Mermin entropy of smeared subsystems) and F_fde = E_fde - TS.  E_xc_nad and E_H_nad are
 * the nonadditive parts E[rho] - sum_I E[rho_I].  E_band_form is E_fde evaluated by the
 * band-energy ("deband") recast of the Appendix from the stored eigenvalues.  iters is the
 * number of inner iterations the call made; dE the last energy change. */
typedef struct {
  double E_fde, F_fde, TS;
  double E_kin, E_nl, E_loc, E_H, E_xc, T_nad, E_xc_nad, E_H_nad, E_nn;
  double E_band_form;
  int iters;
  double dE;
} fde_energies;

/* Create a context on the current CUDA device.  cuda_stream is a cudaStream_t (NULL: the
 * legacy default stream).  Errors: FDE_EINVAL (null/invalid descriptor), FDE_EUNSUPPORTED
 * (non-orthorhombic cell, grid sizes), FDE_ENOMEM/FDE_ECUDA. */
fde_status fde_create(const fde_cell_desc* cell, const fde_func_desc* func, fde_prec prec,
                      void* cuda_stream, fde_ctx** out);

/* Add a subsystem (copies every host array); builds its plane-wave spheres, FFT column
 * maps and projector tables on the device.  *sub_id receives its index (0, 1, ...).
 * The first call also fixes the set of atoms grouped in the all-nuclei local potential;
 * adding subsystems after fde_build_vemb has run returns FDE_EINVAL. */
fde_status fde_add_subsystem(fde_ctx* ctx, const fde_subsys_desc* desc, int* sub_id);

/* Number of plane waves of (sub, k) and, if h_miller is not NULL, their Miller indices
 * [npw][3] (host int) in the library's order. */
fde_status fde_get_basis(fde_ctx* ctx, int sub, int k, int* npw, int* h_miller);

/* Set the density rho_I of a subsystem from a real grid [n1][n2][n3] (FP64).  on_device:
 * 1 if rho is a device pointer, 0 if host. */
fde_status fde_set_density(fde_ctx* ctx, int sub, const double* rho, int on_device);

/* Copy rho_I (sub >= 0) or rho = sum_I rho_I (sub = -1) to a caller device buffer. */
fde_status fde_get_density(fde_ctx* ctx, int sub, double* d_rho);

/* Recast effective potentials of every subsystem (Appendix, recast effective potential):
 * V_eff^I = V_eN (all nuclei) + V_H[rho] + V_XC[rho_I] + V_XC^nad + V_kin^nad
 *         = v_loc + v_H[rho] + v_xc[rho] + v~_kin[rho] - v~_kin[rho_I],
 * with rho = sum_I rho_I (Eq. meth:1), v_H(G) = 4 pi rho(G)/|G|^2 (FFT Poisson solve),
 * GGA gradients and divergences through FFTs and v~_kin from the Appendix's GGA derivative.
 * Stored in the context for fde_apply_h.  d_veff_out (nullable): device [nsub][N_r] FP64
 * copy.  e (nullable, synchronising): receives the grid energy terms E_loc, E_H, E_xc,
 * T_nad, E_xc_nad, E_H_nad, E_nn (the orbital terms are left 0). */
fde_status fde_build_vemb(fde_ctx* ctx, double* d_veff_out, fde_energies* e);

/* Overwrite V_eff^I of one subsystem with a caller grid (device, FP64) -- for tests and
 * for callers that build their own potentials. */
fde_status fde_set_veff(fde_ctx* ctx, int sub, const double* d_veff);

/* H_I psi for a block of nb orbitals of (sub, k) (Eq. KS with the nonlocal projectors of
 * the atoms of I only, Appendix):
 *   (H psi)(G) = |k+G|^2/2 psi(G) + P_sphere FFT[V_eff^I(r) . IFFT psi](G)
 *              + sum_{a in I} sum_ij beta_ai(k+G) D_ij <beta_aj|psi>.
 * d_psi, d_hpsi: device [nb][npw] complex, double2 in FDE_PREC_FP64 contexts and float2 in
 * FDE_PREC_MIXED contexts; they must not overlap.  Asynchronous on the context stream. */
fde_status fde_apply_h(fde_ctx* ctx, int sub, int k, const void* d_psi, void* d_hpsi, int nb);

/* The subsystem's overlap S_I psi = psi + sum_{a in I} sum_ij beta_ai q_ij <beta_aj|psi> for a block
 * of nb orbitals of (sub, k) (Appendix: subsystem-specific PAW / ultrasoft projectors; a copy of
 * psi for norm-conserving subsystems).  Layout and precision as fde_apply_h; asynchronous. */
fde_status fde_apply_s(fde_ctx* ctx, int sub, int k, const void* d_psi, void* d_spsi, int nb);

/* Same as fde_apply_h with host buffers (complex double [nb][npw] in both precisions);
 * synchronising.  Page-locked buffers (cudaHostAlloc, cudaMallocHost or cudaHostRegister) are
 * copied directly by the copy engines; pageable ones go through a page-locked staging buffer
 * of the context (an extra host copy each way). */
fde_status fde_apply_h_host(fde_ctx* ctx, int sub, int k, const double* h_psi, double* h_hpsi,
                            int nb);

/* H psi for every band of every (subsystem, k) of the context's stored orbitals, written
 * into the context's H psi buffers: one batched pass of the hot path.  Asynchronous. */
fde_status fde_apply_h_all(fde_ctx* ctx);

/* One pass of the hot path over the whole cell: fde_build_vemb (no energies) followed by
 * fde_apply_h_all.  use_graph = 1 replays the pass from a CUDA graph captured on the
 * context stream (captured on the first call, and again whenever the context has
 * reallocated device memory since); the context stream must then not be the legacy default
 * stream (FDE_EINVAL).  Asynchronous. */
fde_status fde_hot_step(fde_ctx* ctx, int use_graph);

/* fde_hot_step with host buffers, the end-to-end form of the hot path: h_rho[nsub] the
 * subsystem densities (double [N_r], grid order), h_psi[nblocks] the orbital blocks and
 * h_hpsi[nblocks] their H psi (complex double [nbands][npw]), one block per (sub, k) in
 * subsystem-major, k-minor order.  The orbital blocks go up on a copy stream of the context
 * while the densities go up and the potentials are built on the context stream; every band
 * then goes through the batched H psi and the results come back block by block.  The blocks
 * replace the stored orbitals (their eigenvalues are dropped).  Page-locked host buffers are
 * copied by the copy engines directly (pageable ones work, without overlap).  Synchronising. */
fde_status fde_hot_step_host(fde_ctx* ctx, const double* const* h_rho, const double* const* h_psi,
                             double* const* h_hpsi);

/* Copy the stored H psi of (sub, k) (written by fde_apply_h_all / fde_hot_step and by the
 * eigensolver) to a caller device buffer, complex double [nbands][npw].  Synchronising. */
fde_status fde_get_hpsi(fde_ctx* ctx, int sub, int k, double* d_hpsi);

/* Initial orbitals of (sub, k) from raw complex draws h_raw [nbands][npw][2] (host):
 * c_G = raw_G / (1 + |k+G|^2/2), then orthonormalised on the device. */
fde_status fde_init_orbitals(fde_ctx* ctx, int sub, int k, const double* h_raw);

/* Replace / read the stored orbitals of (sub, k): device complex double [nbands][npw].
 * h_eig, h_occ (nullable): host [nbands] eigenvalues and occupations.  fde_set_orbitals is
 * asynchronous on the context stream: d_psi must stay valid (and unchanged) until the stream
 * has consumed it (fde_sync); fde_get_orbitals synchronises. */
fde_status fde_set_orbitals(fde_ctx* ctx, int sub, int k, const double* d_psi);
fde_status fde_get_orbitals(fde_ctx* ctx, int sub, int k, double* d_psi, double* h_eig,
                            double* h_occ);

/* Block Davidson on (sub, k) with the current V_eff^I (Eq. KS): refines the stored orbitals
 * and eigenvalues until every band's residual norm |H psi - eps psi| < tol or max_iter
 * iterations.  *iters (nullable) receives the iteration count.  FDE_ENOCONV if not
 * converged (the best orbitals are kept). */
fde_status fde_subspace_solve(fde_ctx* ctx, int sub, int k, double tol, int max_iter,
                              int precond, int* iters);

/* Occupations of subsystem sub from its stored eigenvalues (Fermi-Dirac with bisection
 * for the chemical potential, or integer filling), then rho_I = 2 sum_k w_k sum_j n_jk
 * |u_jk|^2 (Sec. 2) from the stored orbitals.  The new density replaces rho_I. */
fde_status fde_update_density(fde_ctx* ctx, int sub);

/* ---- learned preconditioner of the block eigensolver (no counterpart in the paper, which
 * leaves the eigensolver to its host code; Eq. KS is what the solver solves).
 * The preconditioned residual is W_jG = K(y) exp(o_jG) R_jG with K the Teter-Payne-Allan
 * factor, y = (|k+G|^2/2) / T_j (T_j the band's kinetic energy) and o the output of a per-G
 * network: three tanh layers of width 64 and a linear output on the features
 * (log(1 + y), log T_j, |R_jG| / rms_G |R_j|).  Parameters: FDE_PRECOND_PARAMS floats,
 * W1[64][3] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4.  Inference uses the
 * weights rounded to bfloat16 with FP32 accumulation: the two 64 x 64 layers as BF16
 * tensor-core MMAs (activations split into two bf16 terms, ~2^-18 relative; the default) or
 * on the CUDA cores (fde_set_precond_path); training keeps FP32 master weights (split into two
 * bf16 terms for the tensor-core forward, back-propagation and weight-gradient products).
 * Training pairs (R, D): D the ideal correction of residual R.  The loss is
 * sum_j sum_G |m_jG R_jG - D_jG|^2 / |D_j|^2; training takes full-batch Adam steps. */
/* Where the learned preconditioner's inference and training kernels run, process-wide:
 * 1 tensor cores (default), 0 CUDA cores.  FDE_EINVAL for other values. */
fde_status fde_set_precond_path(int path);
fde_status fde_set_precond(fde_ctx* ctx, int precond); /* preconditioner of fde_scf_subsystem /
                                                          fde_freeze_thaw_cycle solves */
fde_status fde_precond_set_weights(fde_ctx* ctx, const float* h_params);      /* resets Adam */
fde_status fde_precond_get_weights(fde_ctx* ctx, float* h_params, float* h_bf16_rounded);
/* Pairs from the converged orbitals of (sub, k): h_raw [n][npw][2] seeded raw draws, shaped by
 * 1/(1 + |k+G|^2/2), orthogonalised to the converged block and normalised into D; then
 * R = (H - eps_j) D_j for the first n bands.  Needs a converged fde_subspace_solve. */
fde_status fde_precond_harvest(fde_ctx* ctx, int sub, int k, const double* h_raw, int n);
/* Caller pairs: h_r, h_d complex double [n][npw] (host), h_tband [n] band kinetic energies. */
fde_status fde_precond_add_pairs(fde_ctx* ctx, int sub, int k, int n, const double* h_r, const double* h_d,
                                 const double* h_tband);
/* Pairs from the eigensolver's own iterations: while iterations > 0, every fde_subspace_solve
 * (and every solve inside an SCF) keeps (R, X) of its first `iterations` iterates and, once
 * it converges to the block Psi, stores the pairs (R, (1 - Psi Psi^H) X): the error of each
 * iterate is the correction its residual asks for.  0 stops recording. */
fde_status fde_precond_record(fde_ctx* ctx, int iterations);
fde_status fde_precond_clear(fde_ctx* ctx);
/* Loss and gradient (FP32 master weights) over every stored pair; h_grad [FDE_PRECOND_PARAMS]. */
fde_status fde_precond_loss_grad(fde_ctx* ctx, double* h_grad, double* loss);
fde_status fde_precond_train(fde_ctx* ctx, int steps, double lr, double* loss_first, double* loss_last);
/* W = preconditioned R for nb rows of (sub, k) (device, working-precision complex [nb][npw]),
 * h_tband [nb] band kinetic energies. */
fde_status fde_precond_apply(fde_ctx* ctx, int sub, int k, const void* d_r, void* d_w, int nb,
                             const double* h_tband);
/* Cumulative eigensolver iterations and band-applies of H made by the context. */
fde_status fde_get_stats(fde_ctx* ctx, long long* davidson_iters, long long* hpsi_bands);

/* Every energy term of the current state (synchronising). */
fde_status fde_energy(fde_ctx* ctx, fde_energies* out);

/* Self-consistent field of one subsystem with every other density frozen: repeat
 * {build V_eff^I, Davidson on every k, occupations and density, Pulay mixing} until the
 * FDE free energy changes by less than tol_ha and int|rho_out - rho_in| < 10 tol_ha
 * (mixed-precision contexts: max(10 tol_ha, 1e-4)).
 * out (nullable) gets the energies. FDE_ENOCONV after max_scf iterations. */
fde_status fde_scf_subsystem(fde_ctx* ctx, int sub, double tol_ha, int max_scf,
                             fde_energies* out);

/* One Jacobi freeze-and-thaw cycle (Fig. 1b: each subsystem's SCF runs to self-consistency
 * before the densities are exchanged): every subsystem runs fde_scf_subsystem against the
 * densities frozen at the start of the cycle, then every rho_I is refreshed together.
 * Mixed-precision contexts run the cycle twice: first in the FP32 engine with the subsystem
 * SCFs to max(tol_ha, 1e-5), then in the FP64 engine (created on first use) against the same
 * frozen densities, each subsystem's SCF starting from the FP32 cycle's orbitals and output
 * density, to tol_ha; the FP64 result is copied back to the context's state.
 * out (nullable) receives the energies of the refreshed state. */
fde_status fde_freeze_thaw_cycle(fde_ctx* ctx, double tol_ha, int max_scf, fde_energies* out);

/* SCF of every subsystem with the total density refreshed after every step: the paper's
 * default scheme (Sec. 2, text after Fig. 1; Fig. 1b caption: the subsystem SCF is executed
 * once per exchange of the densities, so at convergence every subsystem density is
 * self-consistent with every other one; freeze-and-thaw cycles repeated to convergence reach
 * the same fixed point).  Each step rebuilds V_eff^I of every subsystem from the current
 * densities, runs the block eigensolver on every (subsystem, k), forms the occupations and
 * output densities, and mixes the densities of all subsystems together (one Pulay step on
 * the stacked densities, history 8, weight 0.3).  Converged when the FDE free energy changes by less than tol_ha between steps
 * and every subsystem's int|rho_out - rho_in| is below 10 tol_ha (mixed contexts: an FP32
 * stage to max(tol_ha, 1e-5), then the FP64 engine from its densities and orbitals to
 * tol_ha).  On return the subsystem densities are the last output densities and out
 * (nullable) holds their energies, iters the number of steps.  FDE_ENOCONV after max_scf
 * steps.  With a single subsystem this is the plain Kohn-Sham SCF of the supersystem. */
fde_status fde_scf_refresh(fde_ctx* ctx, double tol_ha, int max_scf, fde_energies* out);

/* Number of misplaced electrons <Delta rho> = 1/2 int |rho(r) - rho_ref(r)| dr (Computational
 * Details, Eq. deltarho) between the context's total density rho = sum_I rho_I and a caller
 * device grid d_rho_ref (FP64 [n1][n2][n3], e.g. the density of a supersystem Kohn-Sham
 * context on the same cell and grid); synchronising. */
fde_status fde_delta_rho(fde_ctx* ctx, const double* d_rho_ref, double* out);

/* Per-kernel timing of the library's own launches (measurement support; no counterpart in
 * the paper).  fde_profile_enable(ctx, level) clears the records and starts recording a
 * CUDA event pair around launches on the context stream: level 1 the three passes of the
 * local H psi (k_zinv, k_plane, k_zfwd), level 2 also the potential build (k_fft_axis_f64 /
 * k_fft_axis_f32, k_unpack_density, k_pw_total, k_pw_pair, k_assemble_pair, k_finish_pair,
 * k_pack2, k_combine, k_nonfinite), the band-block products (k_gemm_hn_tc, k_gemm_rot_tc,
 * k_gemm_hn_partial, k_gemm_hn_reduce, k_gemm_rot, k_kb_couple) and the density passes
 * (k_zinv_density, k_plane_density); 0 stops.  FDE_EINVAL for other levels.
 * fde_profile_get returns the number of recorded launches of `kernel` and their summed
 * device time in ms (synchronising; 0 launches if none). */
fde_status fde_profile_enable(fde_ctx* ctx, int enable);
fde_status fde_profile_get(fde_ctx* ctx, const char* kernel, int* launches, double* total_ms);

/* Number of CUDA kernel launches the context's calls have made since it was created
 * (counted on the host at every launch; measurement support, no counterpart in the paper). */
fde_status fde_launch_count(fde_ctx* ctx, long long* launches);

/* Local part of H psi without any device allocation, for callers that cannot call
 * cudaMalloc (code running under another framework's memory pool or allocator hooks, a
 * host application that owns every device allocation, or a call path that must not grow
 * the device footprint).  The paper has no counterpart: this is a deployment variant of
 * the local part of fde_apply_h, (H psi)(G) = |k+G|^2/2 psi(G) + P_sphere FFT[v . IFFT psi],
 * without the nonlocal projectors and without a context.
 *   cell:     orthorhombic cell and grid (ecut_ha unused); kfrac: host k-point [3], crystal.
 *   d_miller: device int [npw][3], the sphere in the library's order (fde_get_basis).
 *   d_veff:   device double [n1][n2][n3]; d_psi, d_hpsi: device complex double [nb][npw],
 *             not overlapping.  cuda_stream: cudaStream_t (NULL: legacy default stream).
 * Working memory is a set of fixed device arrays inside the library (about 26 MB, held by
 * every GPU that loads the library until the process exits); limits: npw <= 65536,
 * ncol <= 8192 (m1, m2) columns, n3 x ncol <= 1048576, n1, n2 <= 160, n3 <= 320,
 * n1 n2 n3 <= 1048576; larger inputs return FDE_EUNSUPPORTED (the column limits are known
 * only after the sphere has been read on the device, so those two come after one stream
 * synchronisation).  Bands are processed in chunks that fit the arrays.  d_miller is
 * checked on the device: (m1, m2) strictly increasing from column to column, m3 contiguous
 * within a column, every m3 in [-n3, n3), no column longer than n3 and m1, m2 spans within
 * n1, n2; a list that breaks any of these returns FDE_EINVAL and writes nothing to d_hpsi.  The first
 * call on a device resolves the arrays' device addresses (cudaGetSymbolAddress).  Calls share
 * the arrays: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the caller.  The call
 * synchronises the stream once (to read the column count).  Errors: FDE_EINVAL (null or
 * non-positive arguments, a sphere list that fails the checks above), FDE_EUNSUPPORTED
 * (sizes above the limits, non-orthorhombic cell, grid sizes not of the form 2^a 3^b 5^c),
 * FDE_ECUDA. */
fde_status fde_apply_h_local_static(const fde_cell_desc* cell, const double* kfrac, int npw, const int* d_miller,
                                    const double* d_veff, const double* d_psi, double* d_hpsi, int nb,
                                    void* cuda_stream);

/* The library's full-grid 3D transform applied in place to a caller grid (complex, [n1][n2][n3],
 * double2 in FP64 contexts and float2 in mixed ones): sign -1 forward, scaled by 1/N_r
 * (f(G) = (1/N_r) sum_r f(r) e^{-iG.r}); sign +1 inverse, unscaled.  Exposed so the
 * transforms can be checked on their own. */
fde_status fde_fft3d(fde_ctx* ctx, void* d_data, int sign);

/* The potential build's 3D transform of an FP64 grid (complex double [n1][n2][n3], in place,
 * scaled as fde_fft3d) in either arithmetic the library uses for it: arith 0 native FP64 (FP64
 * contexts), 1 double-float (two floats per value, about 48 significant bits, on the FP32
 * pipes; mixed contexts transform the densities and their gradients this way).  Exposed so
 * the transforms can be checked on their own. */
fde_status fde_fft3d_f64(fde_ctx* ctx, double* d_data, int sign, int arith);

/* The FP64 Hermitian eigensolver of the Rayleigh-Ritz step applied to a caller matrix:
 * d_A device complex double [n][n] (Hermitian, row-major, not modified), d_w device [n]
 * receives every eigenvalue in ascending order, d_V device complex double [n][n] receives
 * in column j (V[r*n + j]) the unit eigenvector of w[j] for j < nvec and zeros beyond.
 * Householder tridiagonalisation, bisection and inverse iteration; n <= 1024. */
fde_status fde_dense_eigh(fde_ctx* ctx, int n, const double* d_A, int nvec, double* d_w, double* d_V);

/* The band-block inner product C = A^H B of the eigensolver's Gram and subspace-Hamiltonian
 * matrices and of the projector contraction <beta|psi> (Eq. KS; Appendix, projectors),
 * applied to caller data: d_A device complex float [m][lda], d_B [n][ldb] (rows of length
 * K <= lda, ldb), d_C device complex double [m][ldc] receives the m x n result (FP32
 * products, summed over K-chunks in FP64 in a fixed order).  path: 0 CUDA cores (FP32
 * fused multiply-add); 1 tensor cores (tcgen05, TF32 operands, FP32 accumulation);
 * 3 tensor cores with each operand split into TF32 hi + lo parts (hi*hi + hi*lo + lo*hi,
 * FP32 accuracy).  Synchronising; FDE_ETIMEOUT if a tensor-core wait ran out. */
fde_status fde_gemm_hn_f32(fde_ctx* ctx, const void* d_A, int lda, const void* d_B, int ldb, int m, int n,
                           int K, double* d_C, int ldc, int path);

/* The band-block combination Y = alpha sum_i U[i][j] X_i + beta Y of the eigensolver's
 * rotations and of the projector expansion sum_a beta_a (D <beta|psi>)_a (Eq. KS; Appendix,
 * projectors), applied to caller data: d_X device complex float [m][ldx] (rows of length K),
 * d_U device complex double [m][ldu] (n columns used), d_Y device complex float [n][ldy],
 * updated in place (read only when beta != 0).  path as for fde_gemm_hn_f32.  X and Y must
 * not overlap.  Synchronising; FDE_ETIMEOUT if a tensor-core wait ran out. */
fde_status fde_gemm_rot_f32(fde_ctx* ctx, const void* d_X, int ldx, const double* d_U, int ldu, int m, int n, int K,
                            void* d_Y, int ldy, double alpha, double beta, int path);

/* Path (0, 1 or 3, as for fde_gemm_hn_f32) of the FP32 band-block products the library makes
 * in mixed-precision contexts: every inner product (Gram, subspace Hamiltonian, <beta|psi>)
 * and the projector expansion of H psi.  The eigensolver's orbital rotations always use FP32
 * fused multiply-adds (their rounding accumulates in the orbitals), and FP64 products always
 * use the CUDA cores.  Process-wide; the default is 3 (FDE_GEMM_PATH in the environment sets
 * the initial path). */
fde_status fde_set_gemm_path(int path);

/* Poll limit of the waits a tensor-core product makes for each shared-memory stage of its
 * K loop, and of the waits of the learned preconditioner's tensor-core inference for each
 * layer's MMAs (diagnostic support; no counterpart in the paper).  Every device wait of the
 * library is bounded: when a stage wait runs out the kernel stops issuing, waits (with the
 * full bound, about a second) for the MMAs it has issued, releases its tensor memory, writes
 * no result and the call returns FDE_ETIMEOUT.  polls = 0 makes every stage wait run out at
 * once (so that this path can be exercised on a healthy GPU); polls < 0 restores the default
 * bound.  Process-wide, current device.  If a kernel ever cannot confirm its issued MMAs
 * complete it keeps its tensor memory (an MMA may still write it), and every later product
 * in the process runs on the CUDA cores. */
fde_status fde_set_tc_wait_limit(long long polls);

/* The FP32 plane pass of H psi (the (x, y) transforms, potential multiply and back) comes in
 * several compiled variants (CTAs per SM, radix order of the line transforms, fused x pass,
 * thread mapping of the row transforms, fused column scatter and gather).  The first large batch of a grid shape times each once on the batch
 * itself and keeps the fastest (measurement support; no counterpart in the paper).  Returns the
 * variant chosen for plane side n1 and z length n3, or -1 if none was tuned yet; the
 * environment variable FDE_PLANE_VARIANT pins one. */
int fde_tuned_plane_variant(int n1, int n3);
/* Pin the plane-pass variant used from now on in this process (0 .. 7; 2 .. 7 fuse the x pass:
 * the inverse transform's last stage, the potential multiply and the forward transform's first
 * stage on the same registers; 4, 5 and 7 map consecutive threads to neighbouring rows in the
 * y transforms; 6 and 7 read the sphere columns straight into the first y stage and write the
 * last y stage's outputs straight back; FP64 plane passes run a pinned 0, 2, 4 or 6 as it is and
 * any other as 0), or return to tuning (-1).  FDE_EINVAL for other values. */
fde_status fde_pin_plane_variant(int variant);

/* ---- host-side numerics (no device work; usable without a GPU) --------------------------
 * The engine's own host routines, exposed so they can be checked and reused anywhere.
 * Cells are orthorhombic: lengths [3] bohr (the diagonal of the lattice).
 *
 * Plane-wave sphere of the subsystem orbitals (Sec. 2, plane-wave expansion; the full
 * sphere): every Miller triple m with |k + G_m|^2 / 2 <= ecut (Ha), evaluated in FP64 from
 * the integer indices, with m1 slowest and m3 fastest (the library's orbital order).  kfrac
 * [3] is the k-point in crystal coordinates.  *npw receives the count; miller (nullable,
 * [npw][3]) and kin (nullable, [npw], |k + G|^2 / 2) are filled when given.  When either is
 * given, *npw must hold on entry the number of entries the buffers have room for (size them
 * with a first call passing NULL for both, which ignores the entry value); a smaller
 * capacity returns FDE_EINVAL with the needed count in *npw and writes nothing.
 * FDE_EINVAL for non-positive lengths or ecut. */
fde_status fde_host_sphere(const double* lengths, const double* kfrac, double ecut, int* npw, int* miller,
                           double* kin);
/* Nuclear repulsion V_NN of Eq. E_FDE: Ewald sum of the point charges Z [natoms] at pos
 * [natoms][3] (bohr) with a uniform neutralising background, into *energy (Ha). */
fde_status fde_host_ewald(const double* lengths, int natoms, const double* pos, const double* Z, double* energy);
/* Occupations (Sec. 2: 2 sum_k w_k sum_j n_jk = N_I) of eig [nk][nb] (Ha) with k weights
 * wk [nk]: sigma > 0 smeared, n = f((e - mu) / sigma) with the chemical potential *mu by
 * bisection to 1e-13 electrons and *ts = sigma S, S = 2 sum_k w_k sum_j s((e - mu) / sigma),
 * for smearing_kind
 *   FDE_SMEAR_FERMI  f = 1 / (1 + e^x), s = -[f ln f + (1 - f) ln(1 - f)] (Mermin);
 *   FDE_SMEAR_GAUSS  f = erfc(x) / 2, s = e^{-x^2} / (2 sqrt(pi));
 *   FDE_SMEAR_MP     first-order Methfessel-Paxton (Computational Details):
 *                    f = erfc(x) / 2 - x e^{-x^2} / (2 sqrt(pi)), s = (1 - 2x^2) e^{-x^2} / (4 sqrt(pi))
 *                    (occupations may leave [0, 1]);
 * sigma <= 0 integer occupation of the nelec/2 lowest bands (nk must be 1), *mu the highest
 * occupied eigenvalue, *ts = 0.  occ [nk][nb] out.  FDE_EINVAL for inconsistent arguments. */
fde_status fde_host_occupations(int nk, int nb, const double* eig, const double* wk, double nelec, double sigma,
                                int smearing_kind, double* occ, double* mu, double* ts);
/* Brillouin-zone sampling (Computational Details: Monkhorst-Pack meshes for the periodic
 * systems, Gamma for molecules).  The q[0] x q[1] x q[2] mesh k_j = (2 r_j - q_j - 1 + shift_j) /
 * (2 q_j), r_j = 1..q_j (crystal coordinates; shift nullable = unshifted) is reduced to one
 * point per orbit under the operations k -> R k for the sign-flip masks ops[nops] (3-bit: bit c
 * flips coordinate c; the identity is implied) and, if time_reversal, k -> -R k (Kramers:
 * e(k) = e(-k), |u_-k|^2 = |u_k|^2, exact without any spatial symmetry).  kpts [nk][3] and wk [nk]
 * (orbit size / mesh size) are filled when given; as for fde_host_sphere, *nk holds their
 * capacity on entry then (NULL for both: only the count).  Points equal modulo a reciprocal
 * lattice vector are one point.  FDE_EINVAL for bad arguments or a short capacity. */
fde_status fde_host_kmesh(const int* q, const double* shift, int time_reversal, int nops, const int* ops, int* nk,
                          double* kpts, double* wk);
/* The sign-flip operations r -> R r about the origin (masks as above, identity first) that map
 * the atoms pos [natoms][3] onto atoms of the same charge Z within tol bohr, modulo the
 * orthorhombic cell lengths [3]: *nops of them into ops [8]. */
fde_status fde_host_symmetry_ops(const double* lengths, int natoms, const double* pos, const double* Z, double tol,
                                 int* nops, int* ops);
/* Symmetrise every density the context builds from orbitals over the group of sign-flip
 * operations ops[nops] (must contain the identity 0, be closed under composition and map each
 * subsystem's atoms onto that subsystem's atoms; else FDE_EINVAL):
 * rho(r) <- (1 / nops) sum_R rho(R r).  With it, subsystems may be given the reduced k-sets of
 * fde_host_kmesh for the same operations.  nops = 1, ops = {0} switches it off. */
fde_status fde_set_symmetry(fde_ctx* ctx, int nops, const int* ops);

/* Pulay (DIIS) coefficients of the subsystem SCF's density mixing (the paper is silent on
 * mixing): c [m] minimising |sum_i c_i R_i|^2 with sum_i c_i = 1, from the residual
 * overlaps overlap [m][m] = <R_i|R_j>.  FDE_ENOCONV (and c = e_m, the newest residual) when
 * the bordered system is singular. */
fde_status fde_host_pulay(int m, const double* overlap, double* coef);

/* Synchronise the context stream and check the device status word. */
fde_status fde_sync(fde_ctx* ctx);

/* Message of the last failing call on this context ("" if none). */
const char* fde_last_error(const fde_ctx* ctx);

/* Release every device and host resource of the context. */
fde_status fde_destroy(fde_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FDE_H */
