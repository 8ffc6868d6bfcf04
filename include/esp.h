/*
 * esp.h - C ABI of the GB300 (sm_103a) long-range step of Ewald summation with
 * prolates (ESP): charge spreading with a PSWF window, one forward 3D FFT, the fused
 * diagonal scaling + energy / 3x3 virial reduction, the inverse FFT and the force
 * gather with the window gradient.
 *
 * Paper: J. Liang, L. Lu, S. Jiang, "Fast Ewald Summation with Prolates for Charged
 * Systems in the NPT Ensemble" (arXiv:2601.00161).  Citations below name its sections
 * and equations.
 *
 * Conventions shared by every entry point
 *  - cell[9]: the cell matrix h of Sec. 2.2 in COLUMN-MAJOR order, i.e. cell[0..2] is the
 *    first cell vector h_1, cell[3..5] is h_2, cell[6..8] is h_3 (Angstrom).  det h > 0.
 *  - Positions are Cartesian (Angstrom), N x 3 row-major; charges N (e).  They may lie
 *    anywhere; they are wrapped into the cell through reduced coordinates s = h^{-1} r.
 *  - Units are Gaussian: energies in e^2/Angstrom, as the paper's 1/r kernel.  Multiply
 *    energies, virials, pressures and forces by the caller's Coulomb constant (for example
 *    332.0637 kcal Angstrom / (mol e^2)) to convert.
 *  - Tensors are 3x3 row-major.  The virial is W = -(dU/dh) h^T at fixed reduced
 *    coordinates (eq. (instheta) without the kinetic term), so P = W / det h.
 *  - Device pointers belong to the caller, must stay valid until the stream has
 *    finished the call, and are read / written on the plan's stream.  The plan owns all
 *    of its internal buffers.  A plan is not re-entrant: one call at a time.
 *  - Every function returns ESP_OK (0) or a negative ESP_ERR_* code, never aborts and
 *    never traps; esp_last_error() then gives a message.  On an error the outputs are
 *    unspecified but the plan stays usable (except after ESP_ERR_CUDA, which reports a
 *    failed CUDA call and leaves the context in whatever state CUDA left it).
 */
#ifndef ESP_H_
#define ESP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ESP_OK = 0,
  ESP_ERR_ARG = -1,       /* bad argument (null pointer, n < 0, P out of range, ...) */
  ESP_ERR_CELL = -2,      /* det h <= 0 or a non-finite cell entry */
  ESP_ERR_GRID = -3,      /* a mode with |k| <= c/r_c would reach |m_d| >= M_d/2 */
  ESP_ERR_SUPPORT = -4,   /* stencil P >= M_d: the window would wrap onto itself */
  ESP_ERR_NONFINITE = -5, /* a position or charge is NaN or Inf (that atom is skipped) */
  ESP_ERR_CUDA = -6,      /* a CUDA runtime call failed */
  ESP_ERR_CUFFT = -7,     /* a cuFFT call failed */
  ESP_ERR_TIMEOUT = -8,   /* reserved: a bounded device wait gave up */
  ESP_ERR_STATE = -9      /* call order: e.g. esp_forces_from_spectrum with no spectrum */
};

/* precision flags for esp_plan */
enum {
  ESP_FP64 = 0,      /* spread / FFT / scale / gather in FP64; pos, q, F are double */
  ESP_FP32 = 1,      /* spread, FFT, gather and per-mode math in FP32; energy and virial
                        sums in FP64; pos, q, F are float unless ESP_IO_F64 is given */
  ESP_IO_F64 = 16,   /* with ESP_FP32: pos, q and F are double */
  ESP_BF16_GRID = 32 /* with ESP_FP32: the potential grid between the inverse transform and
                        the force gather is stored in BF16 (8-bit mantissa); the gather
                        computes in FP32.  Energy and virial are unchanged (they come from
                        the spectrum); forces lose accuracy (Sec. 4.4 variants).  Needs the
                        library's plane transforms and M3 a multiple of 8 (ESP_ERR_ARG) */
};

typedef struct esp_plan_s* esp_plan_t;

/* Results of one evaluation, host doubles. */
typedef struct {
  double energy_recip;      /* U_F, eq. (UF) with the gridded structure factor (Sec. 4.1) */
  double energy_self;       /* U_self = -psi_0(0)/(2 C_0 r_c) sum q^2, eq. (selfen) */
  double energy_bg;         /* U_cb + U_bb for a net charge, eq. (Corr) (0 if neutral) */
  double virial_recip[9];   /* W_F = V P_F, eqs. (UFPree)/(tensoraniso): prefactor +1/(2V^2) */
  double pressure_recip[9]; /* P_F = W_F / V */
  double pressure_bg;       /* isotropic background pressure, Sec. 3.4 (times I) */
  double volume;            /* det h */
  double qsum;              /* sum q (net charge Q) */
  double q2sum;             /* sum q^2 */
} esp_result;

/* Number of doubles in the device accumulator written by esp_step (see there). */
#define ESP_ACCUM_LEN 16

/*
 * esp_plan - build a plan for N atoms in cell h on an M1 x M2 x M3 grid.
 *   grid[3]  M_d >= 2; the real grid is row-major with the third index fastest.  M1 at
 *            most about 8000 (FP32) or 4000 (FP64): the transform along the first axis
 *            keeps a column group in shared memory (ESP_ERR_ARG beyond).
 *   w        stencil width P (grid points per dimension, Sec. 4.3), 3 <= P <= 12, P < M_d.
 *   c        PSWF shape parameter c > 0 (Sec. 3.1; see esp_c_from_tolerance).
 *   alpha    the split radius r_c in Angstrom (Sec. 3.1, eq. (decomposition)); ESP has
 *            no Gaussian alpha, so this argument carries r_c.
 *   precision ESP_FP64 or ESP_FP32 (optionally | ESP_IO_F64).
 *   stream   cudaStream_t to run on (NULL = legacy default stream).
 * Host set-up (FP64, once): psi_0^c by a Legendre-Galerkin eigen-solve, the piecewise
 * polynomial window tables of Sec. 4.3 (Horner, degree chosen to the precision), the
 * radial psi_0 / psi_0' tables for the Fourier kernel (Sec. 4.3), the 1D deconvolution
 * tables 1/what_d(m)^2 (Sec. 4.2), cuFFT plans and all device workspace.
 * Errors: ESP_ERR_ARG, ESP_ERR_CELL, ESP_ERR_GRID, ESP_ERR_SUPPORT, ESP_ERR_CUDA,
 * ESP_ERR_CUFFT.  *out is NULL on failure.
 */
int esp_plan(esp_plan_t* out, const double cell[9], int64_t n, const int grid[3], int w,
             double c, double alpha, int precision, void* stream);

/* NPT: change the cell (same N, grid, P, c, r_c); no allocation.  The spectrum kept for
 * esp_forces_from_spectrum becomes stale.  The host rebuilds the schedule of the transform
 * along the first axis (which columns meet the cutoff sphere) and copies it on the plan's
 * stream after waiting for that stream, so the call must not happen while the stream is
 * being captured.  Errors: ESP_ERR_CELL, ESP_ERR_GRID. */
int esp_set_cell(esp_plan_t plan, const double cell[9]);

/* Change the stream subsequent calls run on. */
int esp_set_stream(esp_plan_t plan, void* stream);

/*
 * esp_step - the whole long-range step on the plan's stream, asynchronous:
 * wrap + bin/sort, spread (eq. (gridding)), forward FFT, fused scaling + reduction
 * (eqs. (diag), (PFfinal)) and, if forces != NULL, the inverse FFT and the gather of
 * eq. (AD) (Appendix C, analytical differentiation).
 *   pos, q    device arrays (N x 3 and N) of the plan's I/O type.
 *   forces    device array N x 3 of the I/O type, original atom order, or NULL.
 *   d_accum   device array of ESP_ACCUM_LEN doubles or NULL (then the plan's own).
 *             On completion: [0] U_F, [1..6] W_F xx yy zz xy xz yz, [7] sum q,
 *             [8] sum q^2, [9] number of skipped non-finite atoms.
 * No host synchronisation.  Errors found on the host only (arguments); a non-finite
 * input is reported through d_accum[9] (and by esp_energy_pressure).
 */
int esp_step(esp_plan_t plan, const void* pos, const void* q, void* forces, double* d_accum);

/*
 * Per-atom variants of the long-range step.  Each runs the step without forces (so the
 * energy and virial of esp_step land in the plan's own accumulator), builds fields from
 * the spectrum, takes their inverse FFTs and reads them at the atoms with the window
 * (not its gradient).  Outputs are device arrays of the I/O type in the input order;
 * atoms with non-finite input are left untouched.  Asynchronous on the plan's stream;
 * the first call allocates 6 spectra and 6 grids and the batched transforms.
 * Errors: ESP_ERR_ARG, ESP_ERR_CUDA, ESP_ERR_CUFFT.
 *
 * esp_forces_ik - forces by ik-differentiation (Appendix C, eq. (rhodiagforce)):
 *     F_i = -(q_i / (V Mtot^2)) sum_g E(g) w(g / M - s_i),  E = inverse FFT of i k G X,
 *     G = F^c / w^2; three inverse FFTs.  Momentum is conserved exactly (sum_i F_i = 0 up
 *     to rounding), energy only to the discretisation error; esp_forces is the analytical
 *     differentiation the paper uses.   forces: N x 3.
 * esp_local_virial - per-atom long-range virial for local pressure profiles (Sec. 4.4,
 *     eqs. (rhodiag), (PinsFind)): W^i = (q_i / (2 V Mtot^2)) sum_g Pi(g) w(g / M - s_i),
 *     Pi = inverse FFT of K X / w^2, K the pressure kernel of eq. (PFfinal) times V;
 *     sum_i W^i = W_F, P^i = W^i / V.   virial: N x 6 as xx yy zz xy xz yz.
 * esp_atom_energy - per-atom Fourier energy U^i = (q_i / (2 V Mtot^2)) sum_g phi(g) w,
 *     phi = inverse FFT of G X; sum_i U^i = U_F (self and background terms not included).
 *     energy: N.
 */
int esp_forces_ik(esp_plan_t plan, const void* pos, const void* q, void* forces);
int esp_local_virial(esp_plan_t plan, const void* pos, const void* q, void* virial);
int esp_atom_energy(esp_plan_t plan, const void* pos, const void* q, void* energy);

/*
 * esp_near - the near (real-space) part of the PSWF split on the GPU (Sec. 3, eq. (UN);
 * forces as in eq. (Fc); pressure as in eq. (PinsN)): every pair and periodic image with
 * |r_i - r_j + h n| <= r_c, u = r / r_c,
 *     N(r) = (1 - phi_0(u)) / r,   F_N(u) = 1 - phi_0(u) + u psi_0(u) / C_0,
 *     U_N = 1/2 sum' q_i q_j N(r),   F_i = sum_j q_i q_j F_N r_ij / r^3,
 *     W_N = 1/2 sum' q_i q_j F_N r_ij (x) r_ij / r^3,
 * r_ij = r_i - r_j - h n.  W_N carries the sign that -(dU_N/dh) h^T gives; eq. (PinsN)
 * prints the opposite one.  No exclusions.  A cell list of the plan's current cell is
 * built on the device every call; with the long-range step it gives the total Coulomb
 * energy U_N + U_F + U_self + U_bg.
 *   pos, q    device arrays N x 3 and N of the I/O type.
 *   forces    device array N x 3 of the I/O type: overwritten (add = 0) or added to
 *             (add = 1, e.g. after an esp_step that wrote the long-range forces there).
 *   d_out     device array of 7 doubles, overwritten: U_N, W_N xx yy zz xy xz yz.
 * Asynchronous on the plan's stream; the first call allocates the cell-list buffers.
 * Atoms with non-finite input are left out.  Errors: ESP_ERR_ARG, ESP_ERR_CUDA.
 */
int esp_near(esp_plan_t plan, const void* pos, const void* q, void* forces, int add,
             double* d_out);

/*
 * esp_cell_gradient - derivative of the long-range energy U = U_F + U_self + U_bg with
 * respect to the cell matrix at fixed Cartesian positions, for automatic differentiation
 * through NPT cell changes (Sec. 2.2, eq. (instheta), with r = h s):
 *     dU/dh = -W h^{-T} + sum_i F_i s_i^T,   s_i = h^{-1} r_i (as given, not wrapped),
 * W = W_F + U_bg I the virial and F the forces of an esp_step that wrote forces.  At
 * fixed reduced coordinates the second term is absent: dU/dh|_s = -W h^{-T}.
 *   pos, forces  device arrays N x 3 of the I/O type: the positions of that esp_step and
 *                the forces it wrote (atoms with non-finite positions are left out).
 *   d_accum      that step's accumulator (NULL: the plan's own).
 *   d_grad       device array of 9 doubles, row-major (d_grad[3 a + b] = dU/dh_ab),
 *                overwritten.
 * Asynchronous on the plan's stream; uses the plan's current cell.
 * Errors: ESP_ERR_ARG, ESP_ERR_CUDA.
 */
int esp_cell_gradient(esp_plan_t plan, const void* pos, const void* forces,
                      const double* d_accum, double* d_grad);

/* Energy and pressure only (Algorithm 1: no inverse FFT, Sec. 4.1).  Synchronises the
 * plan's stream and fills *out.  Keeps the spectrum so that an immediately following
 * esp_forces_from_spectrum needs no second spread / forward FFT.
 * Errors: ESP_ERR_ARG, ESP_ERR_NONFINITE, ESP_ERR_CUDA, ESP_ERR_CUFFT. */
int esp_energy_pressure(esp_plan_t plan, const void* pos, const void* q, esp_result* out);

/* Forces F_i = -dU_F/dr_i into the caller's device array (eq. (AD); the exact gradient of
 * eq. (UFAnal) carries no factor 1/2, U_F being quadratic in the charges).  Device
 * array N x 3 of the I/O type, original order.  Runs the full step.  Asynchronous. */
int esp_forces(esp_plan_t plan, const void* pos, const void* q, void* forces);

/* Forces from the spectrum kept by the last esp_energy_pressure (same pos, q, cell):
 * scaling, inverse FFT and gather only.  ESP_ERR_STATE if no spectrum is kept. */
int esp_forces_from_spectrum(esp_plan_t plan, void* forces);

/* End-to-end call with HOST buffers: copies pos, q (I/O type) to the device, runs the
 * full step, copies forces (may be NULL) back and fills *out (may be NULL).
 * Synchronous.  pos/q/forces may be pageable or pinned host memory; page-locked pos and
 * q are read in place by the binning kernel (no staging copy), others are copied first.
 * Page-locked, 16-byte aligned forces are written by a kernel through their device
 * mapping; other forces buffers receive a copy-engine transfer. */
int esp_compute_host(esp_plan_t plan, const void* pos, const void* q, void* forces,
                     esp_result* out);

/* Convert a device accumulator (ESP_ACCUM_LEN doubles, already copied to the host) into
 * an esp_result for this plan's cell and constants. */
int esp_result_from_accum(esp_plan_t plan, const double accum_host[ESP_ACCUM_LEN],
                          esp_result* out);

/* Copy the plan's real grid (M1*M2*M3 values of the compute type; after esp_energy_pressure
 * the spread charge rho_s, after a step with forces the potential phi) or the half
 * spectrum of that grid (M1*M2*(M3/2+1) complex values, the forward 3D transform of the
 * grid's current content, taken by this call) into a host buffer.  For tests. */
int esp_copy_grid(esp_plan_t plan, void* host_dst);
int esp_copy_spectrum(esp_plan_t plan, void* host_dst);

/* Plan facts: [0] c, [1] r_c, [2] psi_0(0), [3] C_0, [4] lambda_0, [5] window table
 * degree, [6] radial table degree, [7] max window fit error / psi_0(0), [8] max radial
 * fit error / psi_0(0), [9] tiles, [10] tile T1, [11] T2, [12] T3, [13] launches of the
 * library's own kernels per full step (cuFFT's not counted), [14] background constant
 * X = r_c^2/2 - int_0^{r_c} r phi_0, [15] 1 if the library's plane transforms keep only the
 * box of the sphere (0: cuFFT transforms the planes into the full half spectrum), [16], [17]
 * the box (or full) extent in m1 and m2 of the layout k_xfft works on.
 * Writes min(len, 18) values. */
int esp_plan_info(esp_plan_t plan, double* info, int len);

/* Per-stage timing with CUDA events on the plan's stream.  esp_profile(plan, 1) creates
 * the events and records one before and after every stage of each later step;
 * esp_profile_read synchronises the stream and writes the last step's stage durations
 * in ms, in the order: [0] set-up, [1] bin (which also clears the spread grid and writes
 * the atoms straight into their tiles' slots), [2], [3] unused (0), [4] unused (0),
 * [5] spread, [6] forward plane transforms (cuFFT's for grids whose plane transforms do
 * not fit in shared memory), [7] transform along the first axis fused
 * with the scaling and the sums, [8] inverse plane transforms, [9] gather (stages that
 * did not run read 0).  Writes min(len, 10) values. */
int esp_profile(esp_plan_t plan, int enable);
int esp_profile_read(esp_plan_t plan, double* stage_ms, int len);

/* Release the plan (waits for its stream). NULL is accepted. */
int esp_destroy(esp_plan_t plan);

/* Message for the last error of this plan (or of the last failed esp_plan when plan is
 * NULL).  Valid until the next call on the plan. */
const char* esp_last_error(esp_plan_t plan);

/*
 * esp_spread_noalloc - spreading onto the grid as the plan path does it, without any
 * device allocation.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc when they need a spread grid, for instance code that runs
 * under an allocator or memory pool which forbids further device allocations, a runtime
 * with a device-memory budget fixed at start-up, or a loop that must not pay the implicit
 * device synchronisation a cudaMalloc or cudaFree may cost.  It runs the plan path's
 * bin/sort and spread kernels with their scratch (binning counters, binned atoms, the
 * window table, the per-tile charge sums of the fixed-point bound) in one static device
 * array of the library, about 8.7 MB, which every GPU that loads the library holds until
 * the process exits.
 *   cell, grid, w, c, precision: as for esp_plan (no split radius is needed here).
 *   n <= ESP_NOALLOC_MAX_ATOMS, and the grid at most ESP_NOALLOC_MAX_TILES tiles of
 *        8 x 8 x 16 points (8 x 8 x 8 for w > 8); larger inputs return ESP_ERR_ARG.
 *   pos, q     device arrays (N x 3 and N) of the I/O type; grid_out the caller's device
 *              array of M1*M2*M3 values of the compute type, overwritten with rho_s.
 *   stream     cudaStream_t to run on.  Asynchronous; non-finite atoms are skipped.
 * The window table is rebuilt on the host only when (c, w, precision) changes, and reaches
 * the array as a kernel argument, so no host buffer has to outlive the call.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  All calls
 * share the one array and every call starts by clearing the counters it needs, but calls
 * that overlap on the GPU (other streams, other host threads) race on it: serialise them.
 * Errors: ESP_ERR_ARG, ESP_ERR_CELL, ESP_ERR_SUPPORT, ESP_ERR_CUDA (esp_last_error(NULL)).
 */
#define ESP_NOALLOC_MAX_ATOMS 65536
#define ESP_NOALLOC_MAX_TILES 4096
int esp_spread_noalloc(const double cell[9], int64_t n, const int grid[3], int w, double c,
                       int precision, const void* pos, const void* q, void* grid_out,
                       void* stream);

/* PSWF shape parameter c with psi_0^c(1) / psi_0^c(0) = delta (Sec. 5.1 tuning rule,
 * read as a ratio to psi_0(0)), 0 < delta < 1; returns a negative value on bad input. */
double esp_c_from_tolerance(double delta);

/* Pressure seen by a barostat's cell coupling (Sec. 2.2), from a 3x3 row-major pressure
 * tensor P, for example pressure_recip of esp_result plus pressure_bg on the diagonal
 * plus the near part's W_N / det h.  Sec. 2.2 defines each coupling's pressure as minus
 * the derivative of the energy with respect to its cell variables at fixed reduced
 * coordinates; for the potential energy those derivatives are these combinations of
 * P = -(dU/dh) h^T / det h (eq. (instheta)):
 *   ESP_COUPLE_ISO       out[0] = tr P / 3                         (isotropic, eq. (Pins))
 *   ESP_COUPLE_SEMI      out[0] = (Pxx + Pyy) / 2, out[1] = Pzz    (semi-isotropic: the
 *                        lateral area A in the x-y plane and the height L along z)
 *   ESP_COUPLE_ANISO     out[0..2] = Pxx, Pyy, Pzz                 (eq. (diagona))
 *   ESP_COUPLE_FLEXIBLE  out[0..5] = Pxx Pyy Pzz Pxy Pxz Pyz        (eq. (instheta); P is
 *                        symmetric for pair potentials)
 * Returns the number of values written, or ESP_ERR_ARG for a NULL pointer or an unknown
 * mode.  Host only; needs no plan and no GPU. */
enum {
  ESP_COUPLE_ISO = 0,
  ESP_COUPLE_SEMI = 1,
  ESP_COUPLE_ANISO = 2,
  ESP_COUPLE_FLEXIBLE = 3
};
int esp_pressure_coupling(const double P[9], int mode, double* out);

#ifdef __cplusplus
}
#endif

#endif /* ESP_H_ */
