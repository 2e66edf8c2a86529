/*
 * emu.h -- C ABI of the GB300 (sm_103a) particle-in-cell step for the neutrino
 * fast flavour instability (Richers, Willcox, Ford & Myers, arXiv:2101.02745).
 *
 * One box is a 1D periodic grid of nz cells over [0, Lz) with ndir
 * computational particles per cell.  Each particle carries a position z, a
 * unit direction Omega, weights N and Nbar, and two 3x3 Hermitian density
 * matrices rho (neutrino) and rhobar (antineutrino) (Sec. 2.2).  One time step
 * is one classic fourth-order Runge-Kutta step (Sec. 2.3) of Eq. 4 whose
 * right-hand side is: deposit the particles onto the grid (Eq. 5), interpolate
 * back to each particle (Eq. 6), build the self-interaction Hamiltonian and
 * its antineutrino counterpart (Eq. 2 and Sec. 2.1), and form the commutators.
 *
 * Conventions
 *   - FP64 throughout; CGS units.  Hamiltonians are angular frequencies H/hbar
 *     [1/s]; kappa = sqrt(2) G_F / hbar [cm^3/s] is a configuration value.
 *   - Flavour order e, mu, tau.  A Hermitian matrix is stored as 9 reals
 *     (Sec. 2.2 stores only the upper triangle and diagonal):
 *       [ee, mumu, tautau, Re emu, Im emu, Re etau, Im etau, Re mutau, Im mutau].
 *   - Particle arrays are structure-of-arrays: component k of particle p of a
 *     matrix array lives at [k * P + p].
 *   - Particle numbering (the lattice contract): particle p = d * nz + i has
 *     direction d (0 <= d < ndir) and ring index i.  The paper places one
 *     particle per direction at every cell centre (Sec. 3.1) and every particle
 *     moves at constant velocity c Omega (Eq. 4), so all particles of one
 *     direction keep a common offset from their cell centres: particle i of
 *     ring d sits at ((i + 1/2) dz + X_d) mod Lz, i.e. in cell
 *     (i + s_d) mod nz where s_d is the cell of the ring's particle 0.
 *     emu_init_particles establishes this.  The step kernels need only that
 *     every particle lies in the cell its ring index assigns (within 1e-6
 *     cells of that cell's boundary) and that a ring shares one direction;
 *     they report EMU_ELATTICE otherwise.
 *   - Grid potential A (36 x nz, [c * nz + j]): A0 = kappa (n - nbar^*) in
 *     components 0..8, then A_x, A_y, A_z = kappa (f_i - fbar_i^*) in 9..35, so
 *     that H_p = sum_j w_pj (A0_j - Omega_p . A_j)  (Eq. 2, 5, 6).  This is
 *     what emu_deposit returns.  The step itself deposits the traceless part
 *     only (32 x nz: per moment A0, A_x, A_y, A_z the diagonal differences
 *     11 - 22, 22 - 33 and the six off-diagonal reals): the trace of H
 *     commutes with rho and drops out of Eq. 4.
 *   - Moments (72 x nz, [c * nz + j], cm^-3): n (0..8), f_x, f_y, f_z
 *     (9..35), nbar (36..44), fbar_x, fbar_y, fbar_z (45..71)  (Eq. 5).
 *
 * Memory and streams
 *   - The caller owns all device memory: the particle arrays (emu_particles)
 *     and one workspace of emu_workspace_bytes() bytes.  The library allocates
 *     no device memory of its own and never frees caller memory.
 *   - Every call enqueues work on the stream given to emu_bind and returns
 *     without waiting, except the calls that write host memory (on_host = 1),
 *     emu_timestep and emu_sync, which synchronise that stream.
 *   - A box bound to the legacy default stream (which cannot be captured)
 *     captures and replays its CUDA graphs on a blocking stream the library
 *     creates for it; the legacy stream orders that stream's work implicitly
 *     before and after its own.  No device memory is involved.
 *   - Calls on one box must not run concurrently from several host threads.
 *
 * Errors: every function returns EMU_OK (0) or a negative code; the message
 * of the last failure is available from emu_last_error.  Errors found by the
 * kernels (lattice violation, non-finite grid values) are recorded in a word
 * in the workspace and reported by the next synchronising call.
 */
#ifndef EMU_H
#define EMU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMU_OK 0
#define EMU_EINVAL (-1)    /* bad argument: null pointer, size, unsupported option */
#define EMU_ECUDA (-2)     /* a CUDA runtime call failed */
#define EMU_ENUMERIC (-3)  /* a non-finite value appeared on the grid */
#define EMU_ETIMEOUT (-4)  /* a bounded device-side wait (a grid barrier of the fused step) gave up */
#define EMU_ELATTICE (-5)  /* particles violate the lattice contract */

typedef struct emu_box emu_box;

/* Box parameters. */
typedef struct {
  int32_t nz;          /* cells, >= 1 */
  int32_t ndir;        /* particles per cell (directions), >= 1 */
  double Lz;           /* domain length [cm], > 0 */
  double area;         /* transverse cell area [cm^2]; cell volume dV = (Lz/nz) * area */
  double kappa;        /* sqrt(2) G_F / hbar [cm^3/s] (Eq. 2 divided by hbar) */
  double c_light;      /* speed of light [cm/s] */
  double cfl_adv;      /* C of Eq. 7 */
  double cfl_flavor;   /* C_F of Eq. 7 */
  int32_t shape_order; /* particle shape (Sec. 2.2.1): degree 0-3 of the B-spline, 2 = quadratic (the
                          paper's choice); all boxes of a batch use one order */
  int32_t reserved;    /* must be 0 */
} emu_config;

/* Device pointers to the caller's particle arrays (P = nz * ndir entries each
 * unless stated).  Rings share one direction: ox/oy/oz/N/Nbar are per particle. */
typedef struct {
  double* z;       /* [P] position in [0, Lz) [cm] */
  double* ox;      /* [P] direction, x component */
  double* oy;      /* [P] direction, y component */
  double* oz;      /* [P] direction, z component */
  double* N;       /* [P] neutrinos represented (Eq. 8) */
  double* Nbar;    /* [P] antineutrinos represented (Eq. 8) */
  double* rho;     /* [9][P] neutrino density matrices */
  double* rhobar;  /* [9][P] antineutrino density matrices */
  double* acc;     /* [18][P] RK scratch: running sum (rho components, then rhobar) */
  double* stage;   /* [18][P] RK scratch: state of the next stage */
  int64_t P;       /* must equal nz * ndir */
} emu_particles;

/* Bytes of device workspace a box with this configuration needs (grid,
 * moments, per-direction tables, deposit partial sums, error word).
 * Returns a negative code for an invalid configuration. */
int64_t emu_workspace_bytes(const emu_config* cfg);

/* Validate cfg and create a box (host memory only).  *out receives the box. */
int emu_create(const emu_config* cfg, emu_box** out);

/* Attach caller-owned device memory and a CUDA stream (cudaStream_t, may be
 * NULL for the legacy default stream).  The workspace must be at least
 * emu_workspace_bytes(cfg) bytes and 256-byte aligned; it is cleared here. */
int emu_bind(emu_box* box, const emu_particles* parts, void* workspace, int64_t workspace_bytes,
             void* stream);

/* Initialise every particle on the device (Sec. 3.1): particle p = d*nz + j0
 * at the centre of cell j0 with direction d, weights of Eq. 8 from the
 * per-cell inputs, and the initial flavour state of Eq. 9 with perturbation
 * strength alpha, its random numbers drawn from SplitMix64 keyed by
 * (seed, p, draw).  Host arrays: n_nu[nz], n_nubar[nz] [cm^-3],
 * f_nu[nz*3], f_nubar[nz*3] [cm^-3]; dirs[ndir*3] unit vectors or NULL for the
 * midpoint Fibonacci sphere.  A weight that is negative only by rounding is
 * set to 0; a clearly negative weight (|f| > n/3) gives EMU_EINVAL. */
int emu_init_particles(emu_box* box, const double* n_nu, const double* n_nubar, const double* f_nu,
                       const double* f_nubar, const double* dirs, double alpha, uint64_t seed);

/* Copy particle fields in from (set) or out to (get) caller buffers laid out
 * like emu_particles (rho/rhobar as [9][P]).  Any pointer may be NULL to skip
 * that field.  on_host = 1: host pointers; the call returns once the copy is
 * done (it synchronises the box's stream).  0: device pointers.
 * emu_set_particles also takes on_host = 2: host pointers, asynchronous: the
 * copies are enqueued on the box's stream and the call returns at once
 * (pinned host memory lets them overlap other work); the caller keeps the
 * host arrays valid and unchanged until the stream has passed the copies
 * (an event recorded after the call, or a later synchronising call).
 * emu_set_particles re-validates the rings; with positions from host memory
 * or with directions it also chooses the particle layout when the layout is
 * -1 (see emu_set_layout), which synchronises the stream whatever on_host is;
 * with a fixed layout (0 or 1) it does not check. */
int emu_set_particles(emu_box* box, const double* z, const double* ox, const double* oy,
                      const double* oz, const double* N, const double* Nbar, const double* rho,
                      const double* rhobar, int on_host);
int emu_get_particles(emu_box* box, double* z, double* ox, double* oy, double* oz, double* N,
                      double* Nbar, double* rho, double* rhobar, int on_host);

/* Deposit (Eq. 5) of the state `src` (0: rho/rhobar, 1: the RK stage buffer)
 * at positions z + pos_dt * c * Omega_z into the box's grid potential A (see
 * conventions).  If A_out is not NULL, A is also copied there ([36][nz]). */
int emu_deposit(emu_box* box, int src, double pos_dt, double* A_out, int on_host);

/* Interpolate (Eq. 6) the grid potential A of the last emu_deposit to every
 * particle at positions z + pos_dt * c * Omega_z and write H/hbar [1/s]
 * ([9][P], packed Hermitian) to H_out.  The antineutrino Hamiltonian is -H^* (Sec. 2.1). */
int emu_interpolate_H(emu_box* box, double pos_dt, double* H_out, int on_host);

/* One stage s (1..4) of the classic RK4 step of size dt: deposit the stage
 * state, interpolate, form d rho/dt = -i[H, rho] and d rhobar/dt =
 * -i[-H^*, rhobar] (Eq. 4), and update the scratch (acc, stage); stage 4
 * writes the new rho, rhobar and z.  Stages must be called in order 1..4. */
int emu_rk_stage(emu_box* box, int s, double dt);

/* nsteps full RK4 steps of size dt (dt <= 0: the value of emu_timestep).
 * Replays one captured step as a CUDA graph, as emu_batch_step does. */
int emu_step(emu_box* box, int64_t nsteps, double dt);

/* Per-species moments of the current state (Eq. 5, cm^-3) into out
 * ([72][nz], see conventions). */
int emu_moments(emu_box* box, double* out, int on_host);

/* Domain diagnostics of the current state into out[63]:
 *   [0:9)   <|n_ab|>      as a real 3x3 matrix, row-major   (Eq. 10)
 *   [9:18)  <|nbar_ab|>   likewise
 *   [18:27) <|f^x_ab|>    likewise                          (Eq. 10)
 *   [27:36) <|fbar^x_ab|> likewise
 *   [36:45) <n_ab>        packed Hermitian (one snapshot of Eq. B1)
 *   [45:54) <nbar_ab>     packed Hermitian
 *   [54:63) <n_ab - nbar_ab^*> packed Hermitian: the domain-averaged electron
 *           lepton number matrix, conserved by Eq. 4 with this Hamiltonian (Eq. 18).
 * Averages are over cells. */
int emu_diagnostics(emu_box* box, double* out, int on_host);

/* Eq. 7 from the moments of the current state (maximum over cells and
 * diagonal components of n and nbar).  Synchronises. */
int emu_timestep(emu_box* box, double* dt_out);

/* ---------------------------------------------------------------- batches
 * A batch is nbox independent boxes of any sizes (the parameter sweeps of
 * Sec. 4 run many such boxes) advanced together by the same kernel launches.
 * A box created by emu_create is a batch of one.  All arrays of a batch are
 * concatenated box after box: the particles of box b occupy
 * [poff_b, poff_b + nz_b * ndir_b) of every emu_particles array (poff_b = sum of
 * the earlier boxes' particle counts; particle (d, i) of box b is
 * poff_b + d * nz_b + i; component k of a matrix array at [k * Ptot + p]); grid
 * columns likewise with cell offsets coff_b.  emu_bind, emu_set/get_particles,
 * emu_moments (72 x total cells), emu_sync and the timing calls work on batches;
 * the calls that take one dt or return one value (emu_init_particles,
 * emu_deposit, emu_interpolate_H, emu_rk_stage, emu_step, emu_timestep,
 * emu_diagnostics) need a batch of one. */

/* Totals of a batch: particles, cells, workspace bytes (negative on error). */
int64_t emu_batch_particles(const emu_config* cfgs, int32_t nbox);
int64_t emu_batch_cells(const emu_config* cfgs, int32_t nbox);
int64_t emu_batch_workspace_bytes(const emu_config* cfgs, int32_t nbox);

/* Create a batch from nbox configurations (host memory only). */
int emu_batch_create(const emu_config* cfgs, int32_t nbox, emu_box** out);

/* emu_init_particles for every box (Sec. 3.1, Eq. 8, 9): host arrays
 * n_nu, n_nubar [total cells], f_nu, f_nubar [3 x total cells] (box after
 * box), dirs [3 x total directions] or NULL (Fibonacci sphere in every box),
 * alpha and seed [nbox].  The random draws of box b are keyed by its local
 * particle numbers, so a box initialises as it would alone. */
int emu_batch_init_particles(emu_box* box, const double* n_nu, const double* n_nubar, const double* f_nu,
                             const double* f_nubar, const double* dirs, const double* alpha,
                             const uint64_t* seed);

/* Eq. 7 for every box from its current state; dt_out [nbox] (may be NULL).
 * The results become the boxes' step sizes.  Synchronises. */
int emu_batch_timestep(emu_box* box, double* dt_out);

/* Set the boxes' step sizes dt [nbox] (each positive). */
int emu_batch_set_dt(emu_box* box, const double* dt);

/* nsteps classic RK4 steps of every box with its own step size (Eq. 7 values
 * unless set), all boxes advanced by the same launches.  Three step forms
 * (emu_set_step_form; emu_autotune picks one):
 *   0  one launch per phase: per step one lattice-shift launch and per stage
 *      one deposit, one deposit combination and one RK-stage launch (13), with
 *      programmatic dependent launch (each waits in hardware for its
 *      predecessor's results, so the next kernel's blocks can be scheduled
 *      while the previous one drains);
 *   1  one persistent cooperative launch per step: the same phases with the
 *      same arithmetic in one kernel whose blocks are all resident, separated
 *      by grid barriers whose waits are bounded (emu_set_barrier_timeout).  A
 *      wait that gives up stops the launch; the next synchronising call
 *      reports EMU_ETIMEOUT, the particle state is then that of an unfinished
 *      step, and later launches run normally.
 *   2  RK stages that deposit (Eq. 5) the state they compute at the next
 *      stage's positions (stage 4: the next step's first stage): per step one
 *      lattice-shift launch and per stage one deposit combination and one
 *      RK-stage launch (9), plus one deposit of the state before the first
 *      step of each call.  Units are 32-cell tiles x directions, tile-major; a
 *      warp sums its deposits per tile over 36 cells (the tile and two on each
 *      side), and the combination adds, per cell, the sums of every tile that
 *      reaches it in a fixed order.  Shape orders 0-2 of the lattice path (1D
 *      boxes); a call whose step sizes have dt c >= 1.9 dz in some box (a ring
 *      could then move two cells between stages) runs form 0 instead.  Its
 *      deposit sums in another order than forms 0 and 1: the results agree
 *      with theirs to rounding and are bitwise reproducible for a fixed grid.
 * Forms 0 and 1 give bitwise the same results for the same grid.  The first
 * call captures one step as a CUDA graph (make that call outside any other
 * stream capture; form 2 captures its first step and a later step) and every
 * step replays it: on the box's stream, or for a box bound
 * to the legacy default stream on a blocking stream the library creates,
 * which the legacy stream orders implicitly before and after its own work.
 * With per-kernel timing on, the kernels are launched directly.  Binding,
 * autotuning, emu_set_grid, emu_set_rk_form, emu_set_step_form,
 * emu_set_deposit_form, emu_set_barrier_timeout and emu_set_oscillation drop
 * the graph. */
int emu_batch_step(emu_box* box, int64_t nsteps);

/* emu_diagnostics of every box: out [nbox][63]. */
int emu_batch_diagnostics(emu_box* box, double* out, int on_host);

/* Autotuner: times trial_steps steps of each candidate launch configuration
 * without changing the particle state (the trial steps write their results
 * into the RK scratch), keeps the fastest for later steps, and reports its
 * index c in *choice_out and the per-step times [ms] of the candidates in
 * ms_out[EMU_AUTOTUNE_CANDIDATES] (either may be NULL; -1 for a candidate
 * that cannot run on this device).  A candidate is a step form
 * (emu_batch_step), a grid of blocks of 256 threads whose warps split the
 * work (the number of particles each warp and block takes follows from it),
 * and the RK stage's tile: 30 cells and two halo lanes per warp (form 0) or
 * 32 cells per warp (form 1):
 *   c = 0..5  one launch per phase, grid {304, 152, 608}[c / 2], RK form c % 2
 *   c = 6..9  one cooperative launch per step, grid {304, 152}[(c - 6) / 2],
 *             RK form c % 2;
 *   c = 10..12  step form 2, grid {304, 152, 608}[c - 10] (its RK stage has
 *             32 cells per warp); -1 where form 2 does not run (3D boxes,
 *             particles anywhere, the cubic shape, dt c >= 1.9 dz);
 *   c = 13..16  one launch per phase, grid 304, RK form c % 2, with the
 *             cluster deposit of 8 (c = 13, 14) or 16 blocks (c = 15, 16;
 *             emu_set_deposit_form 1, 2); -1 for 3D boxes, particles
 *             anywhere and cluster sizes the device cannot run.
 * The deposit's summation order depends on the grid, so results are bitwise
 * reproducible for a fixed grid; step forms 0 and 1 and the RK forms give
 * bitwise the same results, form 2 and the cluster deposit the same to
 * rounding.  Candidates 0-12 keep the per-warp deposit.  Synchronises. */
#define EMU_AUTOTUNE_CANDIDATES 17
int emu_autotune(emu_box* box, int trial_steps, int32_t* choice_out, double* ms_out);

/* Step form of emu_batch_step / emu_step: 0 = one launch per phase, 1 = one
 * persistent cooperative launch per step, 2 = RK stages that deposit the next
 * stage (see emu_batch_step).  Form 1 needs every block of the grid resident
 * at once (at most 2 blocks per SM: 304 on GB300) and a device that supports
 * cooperative launches; form 2 the shape orders 0-2.  Forms 1 and 2 need the
 * lattice path of a 1D box.  Errors: EMU_EINVAL (bad form, grid too large,
 * cubic shape for form 2, step in progress). */
int emu_set_step_form(emu_box* box, int32_t form);

/* Particle layout.  The paper places one particle per direction at every cell
 * centre and moves all at constant velocity (Sec. 3.1, Eq. 4), so every box
 * keeps the lattice contract (see the conventions) and the lattice path
 * runs.  Particles may also sit anywhere, with any direction each (installed
 * by emu_set_particles): the deposit (Eq. 5) and interpolation (Eq. 6) are
 * defined for any positions.  Their path sorts the particles by cell at every
 * stage (a stable radix sort of the library's own), deposits with one warp per
 * cell over its stencil's cells in that order (no float atomics: bitwise
 * reproducible), and runs the RK stage with one thread per particle; it is
 * slower than the lattice path.
 *   layout  0: the lattice path (particles off their sites give EMU_ELATTICE);
 *           1: the path for particles anywhere;
 *          -1 (default): chosen when particles are installed: emu_set_particles
 *              with positions from host memory, or with directions, checks
 *              the contract on the device and synchronises the stream to read
 *              the result (a device-to-device copy of positions alone, such as
 *              a checkpoint of the same box, keeps the path in use; call
 *              emu_set_layout(box, -1) to check again); initialised particles
 *              take the lattice path.
 * emu_get_layout reports the path in use (1 = particles anywhere).  The
 * adjoint calls, the fused step form and 3D boxes need the lattice path.
 * Errors: EMU_EINVAL. */
int emu_set_layout(emu_box* box, int32_t layout);
int emu_get_layout(emu_box* box, int32_t* general);

/* Bound [ns] of every grid-barrier wait of the fused step (default 1e9: far
 * above any phase of a box that fits the GPU).  A wait that exceeds it stops
 * the launch and the next synchronising call returns EMU_ETIMEOUT.  0 makes
 * every wait that has to wait give up at once (for tests of that path).
 * Errors: EMU_EINVAL (negative). */
int emu_set_barrier_timeout(emu_box* box, int64_t ns);

/* Deposit of the step's stages in step form 0 and of emu_rk_stage (Eq. 5;
 * step forms 1 and 2 keep their own): 0 = every warp sums its rings of a tile
 * and writes a partial sum, a second launch adds the partials of each cell
 * (the default); 1, 2 = thread-block clusters of 8 or 16 blocks (64 or 128
 * warps) take one tile at a time, split its rings, add their sums through
 * shared and distributed shared memory and write the potential in the same
 * launch.  The clusters save the second launch and its reads; their summation
 * order depends only on the box and the cluster size, so results are bitwise
 * reproducible and agree with form 0's to rounding.  They run the lattice
 * path of 1D boxes on devices with thread-block clusters (16 blocks: where the
 * device allows clusters beyond the portable size).  Errors: EMU_EINVAL (bad
 * form, a 3D box, particles anywhere, a cluster size the device cannot run,
 * step in progress). */
int emu_set_deposit_form(emu_box* box, int32_t form);

/* Form of the RK stage kernel: 1 = 32 cells per warp, 0 = the halo-lane form
 * (both give bitwise the same results), -1 = chosen by units per warp (the
 * default; emu_autotune and emu_set_grid set it too).  Errors: EMU_EINVAL. */
int emu_set_rk_form(emu_box* box, int32_t form);

/* Set the grid of the step kernels to `blocks` blocks of 256 threads (1..608;
 * the default is 304, two per SM; emu_autotune picks among 152, 304 and 608),
 * for callers that share the GPU with other work.  The blocks' warps split the
 * work, so the choice changes the deposit's summation order (results stay
 * bitwise reproducible for a fixed choice) and whether the RK stage runs with
 * 32 cells per warp (every warp walking at least 8 units) or the halo-lane
 * form (the same results); it drops the RK form emu_autotune chose, and the
 * fused step form if not every block of the new grid could be resident.
 * Errors: EMU_EINVAL. */
int emu_set_grid(emu_box* box, int32_t blocks);

/* Vacuum and matter terms of Eq. 2 (Sec. 2.1): masses m_i c^2 [eV], the mixing
 * angles theta12, theta13, theta23 and phase delta_cp [rad] of the standard
 * three-angle mixing matrix U (the paper does not give a parametrisation),
 * the neutrino energy [erg] (one energy for all particles, Sec. 3), the net
 * electron density n_e [cm^-3] (comoving frame: no lepton flux), and the
 * constants hbar [erg s] and erg per eV. */
typedef struct {
  double mass_eV[3];
  double theta12, theta13, theta23, delta_cp;
  double energy_erg;
  double n_e;
  double hbar;
  double erg_per_eV;
} emu_oscillation;

/* Add the vacuum and matter terms to box `box` (-1: every box of the batch):
 * H = U diag(m_i^2 c^4 / 2E) U^dagger / hbar + kappa n_e diag(1, 0, 0) + H_self
 * for neutrinos and Hbar = (H_vacuum^* - H_matter^*) / hbar - H_self^* for
 * antineutrinos; n_e also enters Eq. 7 as the lepton density.  osc = NULL
 * removes them.  emu_interpolate_H still returns the self-interaction term
 * only.  Invalidates the step sizes of Eq. 7 (call the time-step call again). */
int emu_set_oscillation(emu_box* box, int32_t box_index, const emu_oscillation* osc);

/* ------------------------------------------------------------------ adjoint
 *
 * Discrete adjoint of the RK4 step (Sec. 2.3) for gradients of a loss L on the
 * final moments with respect to the particle weights N, Nbar (Eq. 8) and, by
 * the chain rule through Eq. 8, to the initial densities and fluxes.  The
 * paper computes no gradients: these calls serve sensitivity studies of its
 * instability (growth of <|n_emu|>, Eq. 10; final flavour abundances).
 * The calls work on single boxes and on batches (every box of a batch at
 * once); vacuum and matter terms and all shape orders are included.
 * Adjoint vectors are packed like rho (9 reals per matrix, [k * P + p]) and
 * hold dL/d(packed component): lambda is [18 * P] (rho, then rhobar), gN and
 * gNbar are [P].  All pointers are device pointers, except where on_host says
 * otherwise; calls are asynchronous on the box's stream. */

/* Scratch the adjoint step needs, or EMU_EINVAL: 90 doubles per particle (the
 * stage states y2, y3, two stage adjoints and their running sum) plus the
 * shape weights and traceless grid potential of stages 1-3, kept from the
 * recomputed forward stages (3 x (kept weights per particle + 32 per cell)). */
int64_t emu_adjoint_workspace_bytes(const emu_config* cfg);

/* The same for a batch of nbox boxes. */
int64_t emu_batch_adjoint_workspace_bytes(const emu_config* cfgs, int32_t nbox);

/* Seed at the current state from dmom = dL/d(moments) ([72][nz], the layout
 * emu_moments returns): lambda = dL/d(rho, rhobar) is overwritten, the direct
 * terms dL/dN and dL/dNbar are ADDED to gN and gNbar.  Errors: EMU_EINVAL
 * (NULL pointer, RK step in progress). */
int emu_adjoint_seed(emu_box* box, const double* dmom, double* lambda, double* gN, double* gNbar);

/* One adjoint RK4 step.  The box must hold the state at the START of the
 * step (positions and rho, rhobar, as emu_step(box, 1, dt) would take it).
 * dt > 0: the step size of a single box; dt = 0: every box's own step size
 * (emu_batch_set_dt or a time-step call; the only form a batch takes).
 * On entry lambda = dL/dy_{n+1}; on return lambda = dL/dy_n, and the
 * contributions of this step to dL/dN and dL/dNbar are ADDED to gN, gNbar.
 * The step recomputes its stage states (three forward stages into the RK
 * scratch and adj_ws), then runs the stages backward: per stage a deposit of
 * the stage state (H and shape weights), the transposed commutators, a
 * deposit of the adjoint dL/dH (the self-interaction operator of Eqs. 5-6 is
 * symmetric) and its interpolation.  The particle state is unchanged; the RK
 * scratch (acc, stage) is overwritten.  adj_ws: device, 256-byte aligned,
 * at least emu_(batch_)adjoint_workspace_bytes.  The step is captured as a
 * CUDA graph (as emu_batch_step) and replayed while lambda, gN, gNbar and
 * adj_ws stay the same.  Errors: EMU_EINVAL (dt negative or not finite, dt > 0
 * for a batch, dt = 0 with no step sizes set, NULL or short buffers, step in
 * progress), EMU_ECUDA. */
int emu_adjoint_step(emu_box* box, double dt, double* lambda, double* gN, double* gNbar, void* adj_ws,
                     int64_t adj_ws_bytes);

/* Recorded form of the adjoint step, for boxes where memory is cheaper than
 * recomputation.  emu_adjoint_record_step takes one forward step exactly as
 * emu_step (the state advances) and writes its record: the stage states y2,
 * y3, y4, and the shape weights and grid potential of the four stages
 * (emu_batch_adjoint_record_bytes per step).  emu_adjoint_step_recorded then
 * runs that step's adjoint (as emu_adjoint_step, same results) from the
 * record, with no recomputed stages; the box must hold the state at the
 * START of the step again, and adj_ws needs 54 doubles per particle.  dt as
 * in emu_adjoint_step.  Buffers: device, 256-byte aligned.  Each call is
 * captured as a CUDA graph on first use with its buffers (the record; for the
 * adjoint step also lambda, gN, gNbar, adj_ws) and replayed on later calls
 * with the same buffers (up to 256 graphs per box).  Errors: as
 * emu_adjoint_step. */
int64_t emu_batch_adjoint_record_bytes(const emu_config* cfgs, int32_t nbox);
int emu_adjoint_record_step(emu_box* box, double dt, void* rec, int64_t rec_bytes);
int emu_adjoint_step_recorded(emu_box* box, double dt, const void* rec, double* lambda, double* gN, double* gNbar,
                              void* adj_ws, int64_t adj_ws_bytes);

/* Chain rule through Eq. 8 (N_p = (n_c + 3 f_c . Omega_p) dV / M, c the cell
 * a particle starts on at emu_init_particles): out[8][total cells] =
 * dL/dn_nu, dL/dn_nubar, dL/df_nu (x, y, z), dL/df_nubar (x, y, z) per cell.
 * Works on batches.  Errors: EMU_EINVAL (NULL pointer). */
int emu_weight_gradient(emu_box* box, const double* gN, const double* gNbar, double* out, int on_host);

/* --------------------------------------------------------------- 3D boxes
 *
 * The method on a 3D periodic grid (the paper's runs are 1D; Sec. 5 names 3D
 * runs as future work; Eq. 5 and Eq. 6 are stated for any grid).  A 3D box has
 * nx x ny x nz cells over [0, Lx) x [0, Ly) x [0, Lz), cell index
 * c = (jx * ny + jy) * nz + jz, and ndir particles per cell: particle
 * p = d * C + c0 (C = nx ny nz) starts at the centre of cell c0 with direction
 * d.  Its shape is the tensor product of the 1D shape of order shape_order on
 * each axis (w_pj = product of the three 1D weights), the cell volume is
 * dx dy dz, and Eq. 7 takes the smallest cell edge.  The lattice contract of
 * 1D holds on every axis: the particles of a direction keep a common offset
 * from their cells, so particle (d, site) lies in cell site + s_d (mod the
 * cell counts) with one shift per axis; the step kernels report EMU_ELATTICE
 * otherwise.
 *
 * A 3D box is an emu_box created by emu3_create and bound by emu3_bind (which
 * adds the x and y position arrays to emu_particles: z stays in
 * emu_particles).  These calls work on it as on a 1D box: emu_set_particles,
 * emu_get_particles (z, Omega, weights, rho, rhobar), emu_deposit,
 * emu_interpolate_H, emu_rk_stage, emu_step, emu_batch_step, emu_moments
 * ([72][C]), emu_diagnostics, emu_timestep, emu_batch_timestep,
 * emu_batch_set_dt, emu_set_grid, emu_autotune (the one-launch-per-phase
 * candidates), emu_set_oscillation, emu_sync, the timing calls, emu_destroy.
 * The others (the adjoint calls, emu_weight_gradient, the fused step form)
 * return EMU_EINVAL for a 3D box. */
typedef struct {
  int32_t nx, ny, nz;  /* cells per axis, each >= 1 */
  int32_t ndir;        /* particles per cell (directions), >= 1 */
  double Lx, Ly, Lz;   /* domain lengths [cm], > 0 */
  double kappa;        /* sqrt(2) G_F / hbar [cm^3/s] */
  double c_light;      /* speed of light [cm/s] */
  double cfl_adv;      /* C of Eq. 7 (with the smallest cell edge) */
  double cfl_flavor;   /* C_F of Eq. 7 */
  int32_t shape_order; /* 0-3, the 1D shape of every axis (2 = quadratic) */
  int32_t reserved;    /* must be 0 */
} emu3_config;

/* Workspace bytes of a 3D box (negative for an invalid configuration). */
int64_t emu3_workspace_bytes(const emu3_config* cfg);

/* Validate cfg and create a 3D box (host memory only). */
int emu3_create(const emu3_config* cfg, emu_box** out);

/* As emu_bind, plus the device arrays x[P], y[P] of the positions on the x
 * and y axes (caller-owned; P = ndir nx ny nz). */
int emu3_bind(emu_box* box, const emu_particles* parts, double* x, double* y, void* workspace,
              int64_t workspace_bytes, void* stream);

/* Initialise every particle (Sec. 3.1, Eq. 8, 9) as emu_init_particles does,
 * on the 3D lattice: host arrays n_nu[C], n_nubar[C], f_nu[3C], f_nubar[3C]
 * in cell-index order; dirs[3 ndir] or NULL (Fibonacci sphere). */
int emu3_init_particles(emu_box* box, const double* n_nu, const double* n_nubar, const double* f_nu,
                        const double* f_nubar, const double* dirs, double alpha, uint64_t seed);

/* Copy the x and y positions in or out (either may be NULL; on_host as in
 * emu_get_particles).  Setting positions re-validates nothing until the next
 * kernel that checks the lattice. */
int emu3_get_positions(emu_box* box, double* x, double* y, int on_host);
int emu3_set_positions(emu_box* box, const double* x, const double* y, int on_host);

/* Wait for the box's stream and report errors recorded by its kernels. */
int emu_sync(emu_box* box);

/* Kernels launched by this box since creation (for launch accounting). */
int64_t emu_kernel_launches(const emu_box* box);

/* Per-launch device timing.  With enable != 0 every later kernel launch of
 * the box is bracketed by two CUDA events recorded on the box's stream.
 * emu_kernel_times synchronises the stream, writes the summed duration [ms]
 * and the number of recorded launches of each kernel class to ms_out[7] and
 * count_out[7] (0: lattice-shift table, 1: deposit, 2: RK stage, 3: deposit
 * combination, 4: other, 5: fused step, 6: RK stage with the next deposit of
 * step form 2), and clears the record.  Timing is a
 * measurement aid with no other effect. */
int emu_profile(emu_box* box, int enable);
int emu_kernel_times(emu_box* box, double* ms_out, int64_t* count_out);

/* Deposit that allocates nothing (the paper has no counterpart: this is a
 * service for callers of the library).  Some callers cannot call cudaMalloc
 * or any other allocator, yet may still enqueue stream work and wait for it:
 * code inside another library's allocation-free section, or code that must
 * not touch an allocator while a memory pool is being resized or torn down.
 * They cannot provide the workspace emu_bind needs, so this call keeps the
 * deposit's scratch (direction table, lattice shifts, partial sums, error
 * word) in one static 32 MiB device array of the library, which every GPU that
 * loads the library holds until the process exits.
 *   - It must not be called from a host function (cudaLaunchHostFunc or a
 *     stream callback): CUDA forbids CUDA calls there, and this call launches
 *     kernels, copies and synchronises.
 *   - Inputs: cfg and the device particle arrays laid out as in emu_particles
 *     (rho/rhobar as [9][P]); output: A_out, a device array [36][nz] that
 *     receives the grid potential A (as emu_deposit) of the state at positions
 *     z + pos_dt * c * Omega_z.  stream is a cudaStream_t (NULL: legacy stream).
 *     The quadratic shape only (cfg->shape_order 2, else EMU_EINVAL).
 *   - The scratch needs 21 MB of per-warp partial sums, 8.6 KB per 30-cell
 *     tile and 36 bytes per direction; a box that does not fit in 32 MiB
 *     (roughly nz above 43,000 or ndir above 340,000) is rejected with
 *     EMU_EINVAL before any device work.
 *   - The first call on a device looks up the array's device address on that
 *     device (cudaGetSymbolAddress).  No call may be made on a stream that is
 *     being captured: every call ends by copying the error word to the host
 *     and synchronising the stream, which a capture cannot contain; such a
 *     call returns EMU_EINVAL before any device work.  The call clears the
 *     error word, runs the deposit, then synchronises the stream to report
 *     lattice or non-finite errors.
 *   - The address is kept per device for later calls.  After a CUDA error in
 *     a call it is looked up again on the next call; a reset of the device
 *     (cudaDeviceReset) between calls is not supported.
 *   - All calls on a device share the one array, which keeps whatever the last
 *     call left in it: calls that overlap on the GPU (other streams, other host
 *     threads) race on it and must be serialised by the caller.
 * Errors are reported through emu_last_error(NULL). */
int emu_deposit_static(const emu_config* cfg, const double* z, const double* ox, const double* oy,
                       const double* oz, const double* N, const double* Nbar, const double* rho,
                       const double* rhobar, double pos_dt, double* A_out, void* stream);

/* Message of the last failure on this box ("" if none); box may be NULL for
 * failures of emu_create and emu_deposit_static. */
const char* emu_last_error(const emu_box* box);

/* Release the box (host memory only; caller memory is untouched). */
void emu_destroy(emu_box* box);

#ifdef __cplusplus
}
#endif

#endif /* EMU_H */
