/*
 * lbfluct.h -- C ABI of the GB300 fluctuating non-ideal-fluid lattice Boltzmann library.
 *
 * The library advances ensembles of independent periodic lattices with the
 * fluctuating lattice Boltzmann method of Gross & Varnik, "Simulation of static
 * critical phenomena in non-ideal fluids with the Lattice Boltzmann method"
 * (arXiv:1202.4748), Sec. III A:
 *   - evolution equation Eq. 61, moments Eq. 62,
 *   - non-ideal thermodynamics through the pressure tensor Eqs. 63-64: the
 *     modified equilibrium Eq. 65 (LB_MODEQ; the paper's D2Q9 weights, and on
 *     D3Q19 the same structure with the rotation-invariant form of its
 *     square-gradient weights), or a D2Q9/D3Q19 form with the Landau pressure
 *     in the equilibrium and the square-gradient part of the chemical
 *     potential as a Guo body force (LB_GUO),
 *   - collision in the moment basis of Eq. 66 with per-mode relaxation rates,
 *   - local Gaussian noise with the covariance of Eq. 68 (Cholesky-factored),
 *     drawn from a counter-based Philox4x32-10 stream keyed by
 *     (site, step, system, draw) so runs are reproducible and resumable,
 * and accumulates in FP64 the block observables of Sec. II B (Eqs. 46-50) and
 * the structure factor of Eq. 80.
 *
 * Conventions shared by all entry points
 *   Ownership  The caller owns the device workspace (any device allocation of
 *              at least lb_workspace_bytes(), 256-byte aligned) and the CUDA
 *              stream.  The library never allocates device memory.  Host
 *              buffers passed to getters are caller-owned and are not retained.
 *   Errors     Every call returns an lb_status; nothing is thrown across the
 *              ABI.  Device-detected errors (non-positive density, indefinite
 *              noise covariance, non-finite values) are raised by the next
 *              synchronising call (lb_sync, getters) and are sticky: after one,
 *              lb_step returns LB_ERR_STATE until lb_init / lb_write_fields /
 *              lb_load restores a state.
 *   Threads    Thread-compatible: one context per host thread at a time.
 *   Layouts    Host population arrays are float64 [q][nz][ny][nx] (x fastest)
 *              holding f_i(r, t): the populations at site r before the
 *              collision of step t.  Velocity order D2Q9: rest, (1,0), (-1,0),
 *              (0,1), (0,-1), (1,1), (-1,-1), (1,-1), (-1,1).  D3Q19: rest,
 *              +-x, +-y, +-z, then (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0),
 *              (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1),
 *              (0,1,-1), (0,-1,1).
 */
#ifndef LBFLUCT_H
#define LBFLUCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = -1,                 /* invalid argument (sizes, tau, kT, combos)  */
    LB_ERR_CUDA = -2,                /* a CUDA runtime call failed                  */
    LB_ERR_WORKSPACE = -3,           /* workspace too small or misaligned           */
    LB_ERR_NONPOSITIVE_DENSITY = -4, /* rho <= 0 met at some site (device)          */
    LB_ERR_NOISE_NOT_PD = -5,        /* Eq. 68 covariance not positive definite     */
    LB_ERR_NONFINITE = -6,           /* NaN/Inf met in the observables              */
    LB_ERR_UNSUPPORTED = -7,         /* valid but not supported combination         */
    LB_ERR_STATE = -8,               /* sticky error or call out of order           */
    LB_ERR_IO = -9,                  /* checkpoint file error                       */
    LB_ERR_NO_ROOT = -10,            /* a self-consistency equation has no solution  */
    LB_ERR_TIMEOUT = -11             /* a bounded device-side wait ran out            */
} lb_status;

enum { LB_D2Q9 = 0, LB_D3Q19 = 1 };
enum { LB_MODEQ = 0, LB_GUO = 1 };
enum { LB_FP64 = 0, LB_FP32_DEVIATION = 1 };
enum { LB_INIT_UNIFORM_NOISE = 0, LB_INIT_FROM_RHO = 1, LB_INIT_TANH_STRIPE = 2, LB_INIT_FROM_DEVICE_RHO = 3 };
#define LB_MAX_Q 19
#define LB_MAX_LEVELS 32

/* One system of an ensemble.  mu = f0'(phi)/rho_c - kappa lap rho with
 * f0 = a/2 phi^2 + b/4 phi^4, phi = (rho - rho_c)/rho_c (Eqs. 1-3; a, b are
 * the paper's r, u).  tau[a] is the relaxation time of moment a (entries of
 * conserved moments are ignored; every other must exceed 1/2).  The kinematic
 * viscosity of the Holdych term of Eq. 63 uses tau[4] (D2Q9, the c_x^2 - c_y^2
 * mode) or tau[6] (D3Q19, the c_y^2 - c_z^2 mode).  Sizes are >= 1; nz must
 * be 1 for D2Q9.  system_id < 2^24. */
typedef struct {
    int32_t lattice;
    int32_t coupling;
    int32_t nx, ny, nz;
    double rho_c, a, b, kappa;
    double kT;                  /* noise temperature k_B T >= 0 (0: deterministic) */
    double tau[LB_MAX_Q];
    uint64_t seed;              /* Philox key                                       */
    uint32_t system_id;         /* enters the Philox counter                        */
} lb_system_desc;

/* Run options, shared by all systems of a context.  All systems of one
 * context must share lattice, coupling and precision.
 *   precision   LB_FP64 (populations and arithmetic in float64) or
 *               LB_FP32_DEVIATION (float32 populations stored as deviations
 *               from the rest equilibrium f^eq(rho_c, 0) = rho_c on the rest
 *               velocity, float32 collision; observables still FP64).
 *   obs_every   sample the block observables after every obs_every-th step
 *               (time t > 0 with t % obs_every == 0); 0 disables.
 *   sk_every    accumulate C(k) likewise; 0 disables.  Needs equal sides.
 *   graph_chunk if > 0 (even), lb_step replays CUDA graphs of graph_chunk
 *               steps (with the observable launches inside) when the step
 *               counter is a multiple of graph_chunk; 0 = plain launches.
 *   tile        tile shape of the step kernel (0 = library default): (x, y, 1)
 *               on D2Q9; on D3Q19 (x, y, z-chunk) of the z-marching kernel.
 *   occupancy   resident CTAs per SM the step kernel was compiled for (its
 *               register budget); 0 = the tile's default.  Must match a
 *               compiled variant, else LB_ERR_UNSUPPORTED.
 *   variant     if > 0, selects compiled step-kernel variant number
 *               variant - 1 of lb_kernel_variants() directly (overrides
 *               tile and occupancy); 0 = by tile / occupancy / default
 *               (the default's z-chunk adapts to the ensemble, see
 *               lb_kernel_variant).
 *   hist_bins   order-parameter histograms P_L(m) (Sec. II D): every
 *               observable sample also bins each block value m of every
 *               level into hist_bins equal bins on [-hist_range, hist_range)
 *               (plus under/overflow counts); 0 disables, at most
 *               LB_MAX_HIST_BINS.
 *   jk_spectra  1: every structure-factor sample also accumulates the
 *               momentum spectra of lb_momentum_spectra (needs sk_every > 0);
 *               0: off.
 *   hist_range  half-width of the histogram range (> 0 when hist_bins > 0). */
#define LB_MAX_HIST_BINS 4096
typedef struct {
    int32_t precision;
    int32_t obs_every;
    int32_t sk_every;
    int32_t graph_chunk;
    int32_t tile[3];
    int32_t occupancy;
    int32_t variant;
    int32_t hist_bins;
    int32_t jk_spectra;
    double hist_range;
} lb_run_opts;

/* FP64 accumulators of one block level (Eqs. 46-50).  Blocks have dims
 * (bx, by, bz); n counts block samples (blocks x snapshots).  m is the block
 * mean of phi (Eq. 46), e = E_L of Eq. 50 = block mean of phi^2 / 2. */
typedef struct {
    int32_t bx, by, bz, pad;
    double n;
    double sum_m, sum_m2, sum_abs_m, sum_m4, sum_e, sum_e2;
} lb_obs_level;

/* Global FP64 bookkeeping of one system at its latest observable sample. */
typedef struct {
    int64_t step;               /* current step counter of the context           */
    int64_t n_samples;          /* observable snapshots accumulated              */
    double mass0;               /* sum rho at initialisation                     */
    double mass;                /* sum rho at the latest sample                  */
    double momentum[3];         /* sum of sum_i c_i f_i at the latest sample     */
    double rho_mean;            /* mass / sites                                  */
} lb_obs_global;

typedef struct lb_ctx lb_ctx;

/* Bytes of device workspace needed for these systems and options.
 * Errors: LB_ERR_ARG for invalid descriptors (see lb_system_desc). */
lb_status lb_workspace_bytes(const lb_system_desc* systems, int n_systems,
                             const lb_run_opts* opts, size_t* bytes);

/* Create a context over caller-owned device memory d_workspace (bytes long,
 * 256-byte aligned) on CUDA stream `stream` (a cudaStream_t; NULL = legacy
 * default stream) of the current device.  Validates arguments (Sec. III B's
 * low-Mach constraint kT << rho_c/3 is not enforced).  The state is undefined
 * until lb_init, lb_write_fields or lb_load.
 * Errors: LB_ERR_ARG, LB_ERR_WORKSPACE, LB_ERR_UNSUPPORTED, LB_ERR_CUDA. */
lb_status lb_create(const lb_system_desc* systems, int n_systems, const lb_run_opts* opts,
                    void* d_workspace, size_t bytes, void* stream, lb_ctx** out);

/* Initialise every system at step 0 with u = 0 and f = f^eq(rho, 0, grad rho):
 *   LB_INIT_UNIFORM_NOISE  rho = rho_c + amplitude (2U - 1) with U from the
 *                          system's Philox stream (draw 0xFF, step 0), minus its
 *                          FP64 mean so that the average density is rho_c;
 *   LB_INIT_FROM_RHO       rho from h_rho: float64, all systems concatenated in
 *                          descriptor order, each [nz][ny][nx];
 *   LB_INIT_TANH_STRIPE    the two-interface mean-field stripe of
 *                          lb_stripe_density (h_rho and amplitude unused);
 *   LB_INIT_FROM_DEVICE_RHO  as LB_INIT_FROM_RHO with h_rho a device pointer
 *                          (caller-owned, read in stream order on the
 *                          context's stream), so that a caller can stage the
 *                          next input on another stream while the context
 *                          steps.
 * Clears observables and the sticky error.  Synchronises the stream.
 * Errors: LB_ERR_ARG (mode, missing h_rho, a stripe for a system without
 * a < 0 < b), LB_ERR_CUDA. */
lb_status lb_init(lb_ctx* ctx, int mode, double amplitude, const double* h_rho);

/* Mean-field stripe density (host only, no device call), Sec. II A: below the
 * critical point (a < 0, b > 0) the Landau potential has the coexistence
 * densities rho_c +- phi0, phi0 = sqrt(-a/b) (Eq. 20), joined by a tanh
 * interface of width w = sqrt(-2 kappa / a) (Eqs. 22-23).  Writes, for every
 * system in descriptor order ([nz][ny][nx] each, concatenated into out, a
 * caller-owned array of the ensemble's site count), two flat interfaces
 * normal to x at x = nx/4 and 3 nx/4:
 *   rho(x) = rho_c + phi0 (tanh((x - nx/4)/w) - tanh((x - 3nx/4)/w) - 1),
 * the sharp step rho_c +- phi0 when kappa = 0.  Errors: LB_ERR_ARG (null
 * pointers, n < 1, a side < 1, a >= 0, b <= 0 or kappa < 0 in a system). */
lb_status lb_stripe_density(const lb_system_desc* systems, int n_systems, double* out);

/* Advance all systems nsteps time steps (Eq. 61: collide, add noise, stream),
 * sampling observables on the obs_every / sk_every schedule.  Asynchronous
 * on the context's stream.  Errors: LB_ERR_STATE (sticky error / no state),
 * LB_ERR_ARG (nsteps < 0), LB_ERR_CUDA. */
lb_status lb_step(lb_ctx* ctx, int64_t nsteps);

/* Wait for the stream and report device-detected errors. */
lb_status lb_sync(lb_ctx* ctx);

/* Copy the FP64 accumulators of system `sys` (descriptor order) to the host:
 * up to max_levels levels into h_levels (level 0 = whole system, then blocks
 * halving each side while exact, last the single-site level), the level count
 * into *n_levels, and the global bookkeeping into *h_global (nullable).
 * Synchronises.  Errors: LB_ERR_ARG, device errors, LB_ERR_CUDA. */
lb_status lb_observables(lb_ctx* ctx, int sys, lb_obs_level* h_levels, int max_levels,
                         int* n_levels, lb_obs_global* h_global);

/* The accumulators of every system at once (one device-to-host copy of each
 * array and one synchronisation; same content as lb_observables per system).
 * h_levels receives the levels of system 0, then system 1, ... (at most
 * max_levels entries in total); level_first[k] is the index of system k's
 * first level and level_first[n_systems] the total (array of n_systems + 1,
 * filled even when h_levels is too short); h_globals (nullable) receives
 * n_systems entries.  Errors: LB_ERR_ARG (null level_first, or max_levels
 * smaller than the total while h_levels is not null), device errors,
 * LB_ERR_CUDA. */
lb_status lb_observables_all(lb_ctx* ctx, lb_obs_level* h_levels, int max_levels, int* level_first,
                             lb_obs_global* h_globals);

/* Derived quantities of one level at noise temperature kT (Eqs. 47-50):
 * out[0] = M_L = <|m|>, out[1] = chi_L (Eq. 48), out[2] = chi_L low-T form
 * (Eq. 49), out[3] = c_H,L (Eq. 50), out[4] = Binder U_L = 1 - <m^4>/(3<m^2>^2),
 * out[5] = <m>.  Pure host arithmetic.  Errors: LB_ERR_ARG (n == 0, kT <= 0). */
lb_status lb_derive(const lb_obs_level* level, double kT, double out[6]);

/* Order-parameter histogram P_L(m) of level `level` of system `sys` (level
 * order as in lb_observables), accumulated over the obs_every schedule: the
 * histogram of the block values m_L^(b) (Eq. 46) over all blocks and samples
 * (Sec. II D).  Writes nbins + 2 counts to h_counts: [0] values below lo,
 * [1 + k] values in bin k, i.e. with floor((m - lo) * (nbins / (hi - lo))) = k
 * evaluated in float64, [nbins + 1] values at or above hi or NaN; and the
 * range lo = -hist_range, hi = hist_range (nullable).  n_counts must equal
 * hist_bins + 2.  Synchronises.  Errors: LB_ERR_ARG (indices, n_counts),
 * LB_ERR_UNSUPPORTED (hist_bins == 0), device errors, LB_ERR_CUDA. */
lb_status lb_histogram(lb_ctx* ctx, int sys, int level, uint64_t* h_counts, int n_counts, double* lo,
                       double* hi);

/* Estimators of M_L and chi_L from one histogram (Sec. IV, order-parameter
 * distribution), pure host arithmetic.  counts: nbins + 2 values as written by
 * lb_histogram, on a range symmetric about 0 (lo = -hi); vol = L^d, the block
 * volume; kT the noise temperature; bins whose centre has |m| < m_cut are set
 * to zero, also in the normalisation (0 = keep all); frac in (0, 1) bounds the
 * Gaussian-fit window (contiguous bins around the peak with count >= frac x
 * the peak count).  With P_s the histogram symmetrised about m = 0 and k* the
 * first maximum of P_s over bins with centre >= 0:
 *   out[0] m_max  centre of bin k* (M_L as the position of the maximum)
 *   out[1] P_max  P_s(k*) / (N w): N = kept counts + under + overflow, w = bin width
 *   out[2] chi_L  from the peak height: vol / (2 pi kT P_max^2) for a peak in
 *                 the innermost bin (one Gaussian about 0), else
 *                 vol / (8 pi kT P_max^2) (two Gaussians of half weight)
 *   out[3] M_fit  centre of a Gaussian fitted to the peak (weighted least
 *                 squares of log P_s against a quadratic; NaN if the window
 *                 has < 3 bins or is not concave)
 *   out[4] sigma^2 of that Gaussian, out[5] chi_L = vol sigma^2 / kT
 *   out[6] bins in the fit window, out[7] 1 if the peak is central else 0
 *   out[8] <|m|> and out[9] <m^2> over the kept bins (bin centres)
 *   out[10] N.
 * Errors: LB_ERR_ARG (nbins < 2, asymmetric range, vol <= 0, kT <= 0, frac
 * outside (0, 1), null pointers). */
#define LB_HIST_EST 11
lb_status lb_histogram_estimates(const uint64_t* counts, int nbins, double lo, double hi, double vol, double kT,
                                 double m_cut, double frac, double out[LB_HIST_EST]);

/* Structure factor of Eq. 80 accumulated over the sk_every schedule, binned in
 * shells j = 1..nbins (k = 2 pi n / S, shell j holds j(j-1) < |n|^2 <= j(j+1)):
 * h_sum[j-1] = sum over samples and shell points of C(k), h_count[j-1] = number
 * of k points in the shell, *n_samples = snapshots.  Requires equal sides
 * (checked at lb_create) and nbins <= ceil(sqrt(3) S / 2) + 2.  Synchronises.
 * Errors: LB_ERR_ARG, LB_ERR_UNSUPPORTED (sk_every == 0). */
lb_status lb_structure_factor(lb_ctx* ctx, int sys, double* h_sum, int64_t* h_count, int nbins,
                              int64_t* n_samples);

/* Momentum spectra accumulated on the sk_every schedule when jk_spectra = 1
 * (the equilibration check of Sec. III D against Eq. 69, <|j_a(k)|^2> =
 * rho_0 kT): with j = rho u the fluid momentum of the collision (sum_i c_i f_i
 * for LB_MODEQ; plus F/2, F = kappa rho grad lap rho, for LB_GUO), J_a(k) =
 * sum_r j_a(r) exp(-i k.r), N the sites and khat = n / |n| for k = 2 pi n / S,
 * shell j = 1..nbins (as lb_structure_factor) receives
 *   h_sum[0 * nbins + j - 1]  sum of |J_x|^2 / N
 *   h_sum[1 * nbins + j - 1]  sum of |khat . J|^2 / N            (longitudinal)
 *   h_sum[2 * nbins + j - 1]  sum of (|J|^2 - |khat . J|^2) / (N (d - 1))
 *                                                   (transverse, per component)
 * over samples and shell points; h_count and *n_samples as in
 * lb_structure_factor.  Synchronises.  Errors: LB_ERR_ARG, LB_ERR_UNSUPPORTED
 * (jk_spectra == 0), device errors, LB_ERR_CUDA. */
lb_status lb_momentum_spectra(lb_ctx* ctx, int sys, double* h_sum, int64_t* h_count, int nbins,
                              int64_t* n_samples);

/* Ornstein-Zernike fit of a shell-binned structure factor (Eq. 25 with k^2
 * the symbol of the lattice Laplacian, 6 sum_i t_i (1 - cos k.c_i), as the
 * text after Eq. 80 requires), pure host arithmetic.  Inputs: lattice
 * (LB_D2Q9 / LB_D3Q19), side S of the square / cubic system, the shell sums and
 * counts of lb_structure_factor for shells 1..kmax, the number of samples and
 * kT.  With C_j = h_sum / (h_count n_samples) and k2_j the shell mean of the
 * symbol, fits 1 / C_j = a + b k2_j by least squares weighted by
 * h_count C_j^2, and writes out[0] chi = 1 / (kT a), out[1] xi = sqrt(b / a)
 * (NaN unless a > 0 and b >= 0), out[2] a, out[3] b, out[4] shells used.
 * Errors: LB_ERR_ARG (side < 2, kmax < 2, counts that do not match the
 * lattice's shells, non-positive C_j, kT <= 0, fewer than 2 shells). */
lb_status lb_oz_fit(int lattice, int side, const double* h_sum, const int64_t* h_count, int kmax,
                    int64_t n_samples, double kT, double out[5]);

/* ---- Perturbation-theory comparator (Sec. II C) ------------------------------
 * Lattice sums over the wavevectors q != 0 of an S^d periodic lattice (S^2 for
 * LB_D2Q9, S^3 for LB_D3Q19; the momentum integrals of Eqs. 31-32 and 40-42
 * become such sums, the zero mode excluded because the order parameter is
 * conserved), with G(q) = 1 / (m + kappa q^2) and q^2 the symbol of the lattice
 * Laplacian of the simulated model, 6 sum_i t_i (1 - cos q.c_i):
 *   S1 = N^-1 sum_q G,  S1sq = N^-1 sum_q G^2,
 *   S2 = N^-2 sum_{q1, q2} G(q1) G(q2) G(q1 + q2), terms at the zero mode dropped.
 * Evaluated on the device on the caller's stream in a caller-owned device
 * workspace (256-byte aligned, lb_pt_workspace_bytes() long); each call
 * synchronises that stream.  Results are written to host arrays.
 * Errors: LB_ERR_ARG (lattice, S < 2 or N > 2^28, parameters),
 * LB_ERR_WORKSPACE, LB_ERR_CUDA, LB_ERR_NO_ROOT. */
lb_status lb_pt_workspace_bytes(int lattice, int side, size_t* bytes);

/* out[0] S1, out[1] S1sq, out[2] S2 at mass m > 0. */
lb_status lb_pt_sums(int lattice, int side, double m, double kappa, void* d_workspace, size_t bytes,
                     void* cuda_stream, double out[3]);

/* Symmetric phase, Eq. 36: r' = r + 3 u kT S1(r') - 6 u^2 kT^2 S2(r'), the
 * largest root r' > 0 (the branch that tends to r as u -> 0), found by halving
 * from an upper bound where the right side is below r' and bisecting.
 * out[0] r', out[1] chi = 1/r', out[2] xi = sqrt(kappa/r'), out[3] S1(r'),
 * out[4] S2(r').  LB_ERR_NO_ROOT when no r' > 0 solves it. */
lb_status lb_pt_symmetric(int lattice, int side, double r, double u, double kappa, double kT, void* d_workspace,
                          size_t bytes, void* cuda_stream, double out[5]);

/* Broken phase (r < 0, u > 0), Eqs. 40, 42, 43: v from
 * 0 = r + u v^2 + 3 u kT S1(r_sigma), r_sigma = r + 3 u v^2, the root next
 * below the mean-field v^2 = -r/u; then
 * r'_sigma = r_sigma + kT (3 u S1(r_sigma) - 18 u^2 v^2 kT S1sq(r_sigma)).
 * out[0] v, out[1] r_sigma, out[2] r'_sigma, out[3] chi = 1/r'_sigma,
 * out[4] xi = sqrt(kappa/r'_sigma), out[5] S1, out[6] S1sq (at r_sigma).
 * LB_ERR_NO_ROOT when fluctuations leave no ordered solution. */
lb_status lb_pt_broken(int lattice, int side, double r, double u, double kappa, double kT, void* d_workspace,
                       size_t bytes, void* cuda_stream, double out[7]);

/* Copy f_i(r, t) of system `sys` to h_f (float64 [q][nz][ny][nx]).  Synchronises.
 * Errors: LB_ERR_ARG, LB_ERR_CUDA. */
lb_status lb_read_fields(lb_ctx* ctx, int sys, double* h_f);

/* Overwrite f_i(r, t) of system `sys` from h_f (same layout; FP32 contexts
 * round the deviations to float).  Clears the sticky error.  Synchronises.
 * Errors: LB_ERR_ARG, LB_ERR_CUDA. */
lb_status lb_write_fields(lb_ctx* ctx, int sys, const double* h_f);

/* Step counter (number of steps taken since lb_init). */
lb_status lb_get_step(lb_ctx* ctx, int64_t* step);

/* Checkpoint populations, step counter, accumulators and descriptors to a file;
 * lb_load restores them into a context created with identical descriptors and
 * options.  Because the noise is keyed by (site, step, system), a resumed run
 * is bit-identical to an uninterrupted one.  Errors: LB_ERR_IO, LB_ERR_ARG. */
lb_status lb_save(lb_ctx* ctx, const char* path);
lb_status lb_load(lb_ctx* ctx, const char* path);

/* Step-kernel variants compiled for a lattice (LB_D2Q9 or LB_D3Q19): writes up
 * to max_rows rows of LB_VARIANT_COLS int32 (tile x, tile y, tile z or z-chunk,
 * resident CTAs per SM of the register budget (0 = default), producer warps:
 * 0 = every thread stages and collides its own column, > 0 = warp-specialised
 * kernel with that many staging warps, used on the fully relaxed FP32 path;
 * scheme: 0 = tiles or columns whose threads pull the footprint with plain
 * loads, 1 = (D3Q19) producers stage the footprint rows with bulk copies
 * (cp.async.bulk) into shared memory, when every system has nx % 4 == 0,
 * nx >= 8 and all sides >= 3, else the scheme-0 kernel of the same tile runs,
 * 2 = (D2Q9, modified equilibrium only) row-marching strips: one warp per 32
 * sites (x sites per tile) of y rows, densities in registers and warp
 * shuffles, 3 = (paired D3Q19 kernel) producers stage their 16-byte quads of
 * pulled populations in shared memory with cp.async instead of holding them
 * in registers; sites per thread: 1, or 2 = two x-adjacent sites per thread
 * with paired FP32 arithmetic (D3Q19: per consumer thread of the
 * warp-specialised kernel; D2Q9: per lane of 64-site strips, every mode at
 * tau = 1), when the run is FP32 and every system has nx % 4 == 0, else the
 * one-site kernel of the same tile runs)
 * into out (nullable) and returns the number of variants (negative lb_status
 * on error).
 * Row 0 is the default; where the coupling cannot run it (scheme 2 with the
 * Guo form) the first row it can run is.  Selecting a row the coupling cannot
 * run gives LB_ERR_UNSUPPORTED.  Used by the autotuner; no device call. */
#define LB_VARIANT_COLS 7
int lb_kernel_variants(int lattice, int32_t* out, int max_rows);

/* The row of lb_kernel_variants() (0-based) that ctx's step kernel runs.
 * With variant = 0 and no tile or occupancy given, lb_create takes the
 * default row, or a row that differs from it only in a longer z-chunk when
 * the ensemble still has at least twice as many tiles as the GPU holds
 * resident CTAs (fewer halo planes per site, no idle SMs in the last wave).
 * Errors: LB_ERR_ARG. */
lb_status lb_kernel_variant(lb_ctx* ctx, int* row);

/* Host-armed fault injection for testing the error paths without faulting a
 * GPU (the paper has no counterpart).  kind:
 *   LB_FAULT_NONE        disarm;
 *   LB_FAULT_DENSITY, LB_FAULT_NOISE, LB_FAULT_NONFINITE, LB_FAULT_TIMEOUT
 *                        after the step that ends at time at_step, the device
 *                        status word receives the bit a kernel sets on that
 *                        condition (non-positive density, noise covariance not
 *                        positive definite, non-finite observable, timed-out
 *                        wait); lb_sync then reports LB_ERR_NONPOSITIVE_DENSITY,
 *                        LB_ERR_NOISE_NOT_PD, LB_ERR_NONFINITE or LB_ERR_TIMEOUT,
 *                        and the error is sticky as a real one;
 *   LB_FAULT_LAUNCH      lb_step returns LB_ERR_CUDA without launching the step
 *                        that would end at at_step (steps before it run).
 * The fault fires once.  While one is armed, lb_step uses plain launches (no
 * graph replay), so the step is seen on the host.  Errors: LB_ERR_ARG. */
enum { LB_FAULT_NONE = 0, LB_FAULT_DENSITY = 1, LB_FAULT_NOISE = 2, LB_FAULT_NONFINITE = 3, LB_FAULT_TIMEOUT = 4,
       LB_FAULT_LAUNCH = 5 };
lb_status lb_inject_fault(lb_ctx* ctx, int kind, int64_t at_step);

/* Self-test of the bounded device-side waits (the warp-specialised step
 * kernel's hand-offs give up after about 0.3 s instead of hanging): launches one
 * CTA on `cuda_stream` that waits on a shared-memory barrier nothing arrives
 * at, and reads back the status word d_status (one int of caller-owned device
 * memory, zeroed here).  Returns LB_ERR_TIMEOUT when the wait gave up and
 * reported it, as it must; LB_ERR_STATE if the wait completed; LB_ERR_CUDA on
 * a launch or copy error.  The paper has no counterpart. */
lb_status lb_selftest_wait_timeout(int* d_status, void* cuda_stream);

/* Number of kernels this context has launched so far (graph replays count
 * every kernel node).  Instrumentation for benchmarks; no device call. */
lb_status lb_kernel_launches(lb_ctx* ctx, int64_t* count);

/* Largest lattice (sites) that lb_block_moments_noalloc accepts. */
#define LB_NOALLOC_MAX_SITES (1 << 18)

/* Block moments of one density snapshot, for callers that cannot allocate
 * device memory.  The paper has no counterpart: it defines the moments
 * (Sec. II B), not this calling convention.  Callers such as an application
 * whose framework already reserves the whole device memory pool, or a stepping
 * loop that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree, can neither allocate nor provide a scratch workspace; this entry
 * point keeps its scratch in a fixed 6 MiB device array inside the library
 * (held on every device that loads it until the process exits) and allocates
 * nothing, on the device or the host.  Its work lists are built on the device
 * from the lattice shape, so it copies nothing from host memory and does not
 * wait for the stream.
 *   d_rho      device array of rho, float64 [nz][ny][nx] (caller-owned input)
 *   lattice    LB_D2Q9 (2-D blocks, nz must be 1) or LB_D3Q19 (3-D blocks)
 *   d_out      device array of max_levels x 7 float64 (caller-owned output):
 *              per level n, sum m, sum m^2, sum |m|, sum m^4, sum e, sum e^2 of
 *              this one snapshot, levels ordered as in lb_observables, with
 *              phi = (rho - mean rho)/mean rho
 *   n_levels   receives the number of levels (also when max_levels is too small)
 *   d_status   nullable device int (caller-owned): receives 0, or the bit
 *              4 (non-finite) when some moment is NaN or infinite -- the call
 *              itself returns before the device has computed anything, so a
 *              non-finite input shows here, not in the return value
 * Asynchronous on `stream`.  All calls share the library's scratch array, which
 * keeps the previous call's contents (this call clears what it accumulates
 * into): calls that overlap on the GPU race, so order them on one stream.
 * Every call looks up the array's address on the current device; the first
 * call on a device also loads the library's device code there, so make that
 * first call before any stream capture.
 * Errors: LB_ERR_ARG (pointers, sizes, max_levels), LB_ERR_UNSUPPORTED
 * (nx * ny * nz > LB_NOALLOC_MAX_SITES), LB_ERR_CUDA. */
lb_status lb_block_moments_noalloc(const double* d_rho, int nx, int ny, int nz, int lattice, double* d_out,
                                   int max_levels, int* n_levels, int* d_status, void* stream);

/* Release host-side resources (graphs, context); the workspace stays the caller's. */
void lb_destroy(lb_ctx* ctx);

/* Static string for a status code. */
const char* lb_status_string(lb_status status);

/* Library version string. */
const char* lb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBFLUCT_H */
