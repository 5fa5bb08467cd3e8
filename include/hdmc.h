/*
 * hdmc.h -- C ABI of the GB300 hard-disk Monte Carlo library (libhdmc.so).
 *
 * The library runs the massively parallel Monte Carlo (MPMC) method of
 * Anderson, Jankowski, Grubb, Engel and Glotzer, "Massively parallel Monte
 * Carlo for many-particle simulations on GPUs", J. Comput. Phys. 2013, for N
 * hard disks of diameter sigma in a periodic Lx x Ly box, on one NVIDIA
 * GB300 (sm_103a):
 *   - the box is cut into an mx x my grid of cells of width >= sigma that
 *     fall into four checkerboard sets (Sec. 2.1, Eq. 1);
 *   - a sweep shuffles the order of the sets, and for each set lets every
 *     cell of that set shuffle its disks and make n_M trial translations,
 *     rejecting moves that leave the cell or overlap a disk of the 3x3
 *     neighbourhood; it then translates all disks by a random distance
 *     along a random axis direction (a grid shift), which restores
 *     ergodicity (Sec. 2.2, Algorithm 1; Algorithms 2 and 4);
 *   - the pressure comes from the contact value of the pair distribution,
 *     P* = sigma^2 rho (1 + (pi/2) sigma^2 rho g(sigma+)) (Sec. 4, Eq. P).
 *
 * Conventions for every entry point:
 *   - Return value: HDMC_OK (0) or one of the HDMC_E* codes below; a
 *     failing call leaves the handle usable unless it returns HDMC_ECUDA.
 *   - Host pointers are read or written before the call returns; the
 *     library keeps no reference to them.  Device pointers are named so.
 *   - Work is enqueued on the handle's CUDA stream (the legacy default
 *     stream unless hdmc_set_stream was called).  Calls documented as
 *     "synchronises" wait for that stream; the others return after
 *     enqueueing.  Errors raised on the device (cell overflow) are reported
 *     by the next synchronising call.
 *   - A handle is not thread-safe; use one handle per host thread.
 *
 * State layout (for hdmc_get_state/hdmc_set_state and the exported
 * positions): cells are numbered canonically c = cy*mx + cx; each cell has 4
 * slots (a cell narrower than sqrt(2) sigma holds at most 4 disk centres,
 * Sec. 3.1, Fig. 3); slot j of cell c holds a disk iff j < count[c]; a
 * disk's coordinates are stored relative to its cell's lower-left corner
 * (Sec. 3.1, cell-local frames) and lie in [0,wx) x [0,wy).  Unused slots
 * read HDMC_EMPTY_SLOT.  Disks carry no identity: slot order is the order
 * the last shuffle left them in.
 */
#ifndef HDMC_H
#define HDMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define HDMC_OK 0
#define HDMC_EINVAL 1    /* invalid argument or state */
#define HDMC_ECUDA 2     /* a CUDA runtime call failed; the handle should be destroyed */
#define HDMC_EOVERFLOW 3 /* more than 4 disks in one cell */
#define HDMC_EOVERLAP 4  /* two disks closer than sigma */
#define HDMC_ETIMEOUT 5  /* a bounded device wait gave up */
#define HDMC_ENOMEM 6    /* allocation failed or workspace too small */
#define HDMC_ECHECK 7    /* a kernel of a checked build computed a cell index outside the grid */

/* ---- precision of the stored coordinates ---- */
#define HDMC_FP64 0       /* binary64 cell-local offsets; bit-identical to the serial reference */
#define HDMC_FP32_LOCAL 1 /* binary32 cell-local offsets (Sec. 5 stores binary32 coordinates) */

/* ---- cell rule, OR-ed into the precision argument of hdmc_create,
 * hdmc_workspace_bytes, hdmc_strip_create and the batch calls ----
 * By default m = largest even integer <= L/sigma per axis (cells just wider
 * than sigma, about 0.9 disks per cell in a dense fluid).  With
 * HDMC_CELLS_SQRT2, the paper's rule (Sec. 3.1): floor(L/(sqrt(2) sigma))
 * rounded up to the smallest even m > L/(sqrt(2) sigma), the widest cells
 * that still hold at most four centres (Fig. 3; about 1.8 disks per cell).
 * Either way w = L/m with sigma <= w < sqrt(2) sigma; HDMC_EINVAL if the
 * rule gives fewer than 4 cells or cells narrower than sigma. */
#define HDMC_CELLS_SQRT2 0x100

#define HDMC_EMPTY_SLOT (-1.0e4)
#define HDMC_HIST_BINS 200 /* contact histogram: bins of 1e-4 sigma over [sigma, 1.02 sigma) (Sec. 4) */

typedef struct hdmc_handle hdmc_t;

/* Bytes of device memory a handle needs for these parameters (0 if they
 * are invalid).  Memory is 2 copies of the cell state (mx*my cells of 64 B
 * for HDMC_FP64, 32 B for HDMC_FP32_LOCAL) plus a few kilobytes of tables. */
size_t hdmc_workspace_bytes(int64_t N, double Lx, double Ly, double sigma, int precision);

/* Creates a system of N disks (N even, >= 2) placed on a hexagonal lattice
 * of nx x ny sites (ny even, nx*ny = N, the factorisation whose row spacing
 * is closest to sqrt(3)/2 of the column spacing), each displaced uniformly
 * within 0.01 sigma, and binned into the cell grid:
 *   mx = largest even integer <= Lx/sigma (likewise my), wx = Lx/mx,
 *   wy = Ly/my; requires mx, my >= 4, wx, wy < sqrt(2) sigma and
 *   mx*my < 2^32 (cells are indexed in 32 bits on the device).
 * d is the maximum trial displacement (0 < d < min(wx,wy)/2), nselect the
 * number n_M of trial moves per cell and sub-sweep (1..255), seed the key of
 * every random stream.  precision is HDMC_FP64 or HDMC_FP32_LOCAL.
 * dev_workspace: NULL (the library allocates with cudaMalloc and frees in
 * hdmc_destroy) or a device buffer of at least hdmc_workspace_bytes() bytes,
 * 256-byte aligned, owned by the caller, which must outlive the handle.
 * stream: a cudaStream_t or NULL for the legacy default stream.
 * Errors: HDMC_EINVAL (parameters), HDMC_EOVERLAP / HDMC_EOVERFLOW (start
 * not legal), HDMC_ENOMEM, HDMC_ECUDA.  *out is NULL on failure.
 * Synchronises. */
int hdmc_create(hdmc_t **out, int64_t N, double Lx, double Ly, double sigma, double d, int nselect,
                uint64_t seed, int precision, void *dev_workspace, size_t workspace_bytes, void *stream);

/* Replaces the configuration by N disks at the host global coordinates
 * xy[2*i], xy[2*i+1] in [0,Lx] x [0,Ly] (slot order = order of i within a
 * cell).  Resets the grid origin to 0 but keeps the sweep count and the
 * counters.  Errors: HDMC_EINVAL (outside the box), HDMC_EOVERFLOW,
 * HDMC_EOVERLAP; the previous configuration is kept on error.  Synchronises. */
int hdmc_set_positions(hdmc_t *h, const double *xy);

/* Enqueues n sweeps of Algorithm 1: the set order and the shift come from
 * the sweep's own random stream, then 4 sub-sweeps (Algorithm 2) and one
 * cell shift (Algorithm 4).  Sweeps are recorded once into CUDA graphs and
 * replayed.  Returns after enqueueing. */
int hdmc_sweep(hdmc_t *h, int64_t n);

/* Enqueues one extra cell shift (Algorithm 4) drawn from the stream of
 * explicit shifts (independent of the sweeps' streams). */
int hdmc_shift(hdmc_t *h);

/* Enqueues the contact histogram of the current configuration (ordered
 * pairs at distance r in [sigma, 1.02 sigma), bins of 1e-4 sigma, Sec. 4)
 * and adds it to the handle's sample accumulator. */
int hdmc_sample(hdmc_t *h);

/* Pressure from the accumulated samples (one sample of the current
 * configuration is taken first if none were): g(R_i) by Eq. gR at the
 * points R_i of Eq. R, a least-squares polynomial of degree 5 over
 * (sigma, 1.02 sigma] extrapolated to sigma, and Eq. P.  Outputs (each
 * nullable): betaP_over_rho = 1 + (pi/2) rho sigma^2 g(sigma+),
 * g_contact = g(sigma+), hist = the accumulated HDMC_HIST_BINS counts,
 * n_samples = number of configurations accumulated.  Clears the
 * accumulator.  Synchronises. */
int hdmc_pressure(hdmc_t *h, double *betaP_over_rho, double *g_contact, uint64_t *hist, int64_t *n_samples);

/* Bond-orientational order parameter psi_6, the order parameter whose
 * autocorrelation time Sec. 3.3 minimises to tune d and n_M (the paper
 * cites its definition; this is the usual one): the neighbours k of disk j
 * are the other disks closer than r_cut, psi_6(j) = (1/n_j) sum_k
 * exp(6 i theta_jk), computed as z^6 / |z|^6 with z = dx + i dy (0 for a
 * disk without neighbours).  out[0] + i out[1] = the mean of psi_6(j) over
 * the N disks, out[2] = the mean of |psi_6(j)|, out[3] = the mean number of
 * neighbours.  psi (nullable, host, 8*mx*my doubles) receives psi_6(j) of
 * every slot in the layout of hdmc_get_state (real, imaginary; 0 for unused
 * slots); asking for it allocates 64 bytes of device memory per cell for
 * the duration of the call.  0 < r_cut <= 2 min(wx, wy), else HDMC_EINVAL.
 * Synchronises. */
int hdmc_psi6(hdmc_t *h, double r_cut, double out[4], double *psi);

/* Global coordinates of every disk into host xy[2N], in canonical (cell,
 * slot) order: x = O_x + cx*wx + local_x wrapped into [0, mx*wx) (likewise
 * y), O the accumulated grid origin; cells use the binary32 widths in
 * HDMC_FP32_LOCAL mode.  cell (nullable, host int32[N]) receives each disk's
 * canonical cell index.  Synchronises. */
int hdmc_positions(hdmc_t *h, double *xy, int32_t *cell);

/* Raw state in the canonical layout described above: local[(4c+j)*2 + k]
 * (host, 8*mx*my doubles; binary32 values widened exactly) and counts[c]
 * (host, mx*my bytes).  Synchronises. */
int hdmc_get_state(hdmc_t *h, double *local, uint8_t *counts);

/* Restores a raw state taken by hdmc_get_state together with the origin and
 * sweep/shift counters returned by hdmc_info, so that a run can resume
 * bit-identically (the random streams are counter-based).  Values must be
 * representable in the handle's precision.  Synchronises. */
int hdmc_set_state(hdmc_t *h, const double *local, const uint8_t *counts, const double origin[2],
                   uint64_t sweeps_done, uint64_t shifts_done);

/* Snapshots (checkpoint / resume).  The paper does not describe saving a
 * run; because every random draw is addressed by (seed, sweep, cell, set)
 * counters (Sec. 3.2 draws a fresh stream per cell update), the image below
 * determines the rest of the trajectory exactly.
 *
 * A snapshot is a byte image of the complete state of a system in the
 * library's own device layout: a 256-byte header (magic "HDMCSNP1", format
 * version, precision, N, box, sigma, move size d, n_M, grid, seed, balance
 * controls, sweep and shift counters, accumulated sample count), then, each
 * at a 256-byte aligned offset, the device state word (grid origin, next
 * sweep/shift index), the trial counters, the histogram accumulator and the
 * cells (set-major, 4 slots per cell in the handle's coordinate type).
 * Images are portable between hosts of the same byte order.
 *
 * hdmc_snapshot_bytes returns the image size of this handle, or 0 for a
 * NULL handle. */
size_t hdmc_snapshot_bytes(const hdmc_t *h);

/* Writes the snapshot of h into host buf (bytes >= hdmc_snapshot_bytes(h),
 * else HDMC_EINVAL).  Pinned host memory makes the copy asynchronous to the
 * host thread and fast; pageable memory also works.  Returns the device's
 * pending error (HDMC_EOVERFLOW), if any, after writing the image.
 * Synchronises. */
int hdmc_save(hdmc_t *h, void *buf, size_t bytes);

/* Restores a snapshot written by hdmc_save for a system of the same N, box,
 * sigma and precision (d, n_M, seed and the balance controls are taken
 * from the image).  The cells are copied to the device and checked there
 * before anything is replaced:
 * an image with a wrong header, an occupied slot after an empty one, a
 * coordinate outside [0,w) (or NaN), an unused slot not holding
 * HDMC_EMPTY_SLOT, or a disk total other than N is rejected with
 * HDMC_EINVAL and the handle keeps its previous state.  Overlaps are not
 * checked.  Synchronises. */
int hdmc_load(hdmc_t *h, const void *buf, size_t bytes);

/* Cumulative trial counters: out[0] trial moves attempted (n_M per occupied
 * active cell and sub-sweep), out[1] accepted, out[2] rejected because the
 * disk would leave its cell, out[3] rejected because of an overlap.
 * Synchronises. */
int hdmc_counters(hdmc_t *h, uint64_t out[4]);

/* Geometry and progress: cell grid, cell widths (binary64), sweeps and
 * explicit shifts done, grid origin (nullable outputs).  Synchronises. */
int hdmc_info(hdmc_t *h, int32_t *mx, int32_t *my, double *wx, double *wy, uint64_t *sweeps_done,
              uint64_t *shifts_done, double origin[2]);

/* Changes the maximum trial displacement d (0 < d < min(wx,wy)/2) for the
 * sweeps enqueued after this call. */
int hdmc_set_move_size(hdmc_t *h, double d);

/* Balance controls of Table 1 (Sec. 2.4), for negative controls only:
 * shuffle_particles = 0 skips the shuffle of the disks of each cell before
 * its trial moves, shuffle_sets = 0 takes the checkerboard sets in the fixed
 * order 0, 1, 2, 3 instead of a random order per sweep.  Both default to 1
 * (the method); the random streams are consumed as with both on.  Applies
 * to the sweeps enqueued after this call. */
int hdmc_set_balance(hdmc_t *h, int shuffle_particles, int shuffle_sets);

/* Move-size tuning.  d is a free parameter of the method (Sec. 3.3); this
 * sets it for a target acceptance ratio in a pre-run that advances the
 * chain: `sweeps` sweeps in rounds of `every`, after each round
 *   a = accepted / attempted trial moves of the round,
 *   f = sqrt(a / target) limited to [0.5, 2] (2 if nothing was attempted),
 *   d <- d * f limited to [1e-6 sigma, 0.49 min(wx, wy)]
 * (binary64, in this order), then d stays fixed.  The final d is written to
 * d_out (nullable).  0 < target < 1, sweeps >= 1, every >= 1, else
 * HDMC_EINVAL.  Synchronises. */
int hdmc_tune_move_size(hdmc_t *h, double target, int64_t sweeps, int64_t every, double *d_out);

/* Uses stream (a cudaStream_t; NULL = legacy default stream) from now on. */
int hdmc_set_stream(hdmc_t *h, void *stream);

/* Waits for the handle's stream and reports device-side errors. */
int hdmc_sync(hdmc_t *h);

/* Profiling form of hdmc_sweep: runs n sweeps with the same results, but
 * launches every kernel directly (no graph) with a CUDA event pair around
 * it on the handle's stream, and returns the mean device time in
 * milliseconds of one sub-sweep launch, one cell-shift launch and one
 * draws launch (each nullable).  Synchronises. */
int hdmc_profile_sweeps(hdmc_t *h, int64_t n, double *ms_subsweep, double *ms_shift, double *ms_draws);

/* In-step timing: records n sweeps as CUDA graphs of one stage each, as
 * hdmc_sweep records them (programmatic dependent launches), and times
 * their replay with CUDA events on the handle's stream: first the draws and
 * the four sub-sweeps of each sweep without the shifts, then the draws and
 * the shifts alone.  Returns the mean milliseconds per sub-sweep launch and
 * per shift launch inside such a run (each nullable; the draws launch, one
 * per 64 sweeps, is included).  The configuration stays legal, but the
 * trajectory is not that of hdmc_sweep (2n sweep indices are used, sub-sweeps
 * without shifts and shifts without sub-sweeps).  n >= 1, else HDMC_EINVAL.
 * Synchronises. */
int hdmc_profile_stages(hdmc_t *h, int64_t n, double *ms_subsweep, double *ms_shift);

/* ---- spatial decomposition with inactive bands (Sec. 6) -------------------
 * A system split across processors by strips of cell rows.  Strip k of R
 * owns the global rows [r_k, r_{k+1}), r_k = 2 floor(k my / (2R)) (even;
 * every strip has at least two rows, so my >= 2R).  The strip's first row is
 * an inactive band: its cells make no trial moves during the sub-sweeps, so
 * no cell of one strip moves a disk next to a cell another strip moves, and
 * neighbouring strips exchange rows only around the grid shift, which moves
 * the grid (and so the bands) over the disks (Sec. 6 proposes exactly this
 * to cut the communication between processors to once per sweep).  The same
 * chain, serially, is the whole system with those rows inactive.
 *
 * A strip handle holds its rows and two halo rows on either side (rows
 * r_k - 2, r_k - 1 below and r_{k+1}, r_{k+1} + 1 above, periodic) and
 * sweeps in two phases; per sweep, every strip:
 *   1. hdmc_strip_subsweeps: the sweep's draws and its four sub-sweeps;
 *   2. sends its last row (hdmc_strip_get_row which = 3) to the next strip,
 *      which stores it as its halo row r_k - 1 (hdmc_strip_set_halo
 *      which = 1): the shift moves disks of that row into the strip;
 *   3. hdmc_strip_shift: the sweep's grid shift of the strip's own rows;
 *   4. sends its first row (which = 0, the band) to the previous strip, which
 *      stores it as its halo row r_{k+1} (which = 2): the neighbours of that
 *      strip's last row during the next sub-sweeps.
 * The contact histogram (hdmc_sample, then hdmc_strip_histogram) counts the
 * pairs of the strip's own disks and needs all four halo rows current: rows
 * r_k, r_k + 1 (which 0, 1) to the previous strip's halos 2, 3, and rows
 * r_{k+1} - 2, r_{k+1} - 1 (which 2, 3) to the next strip's halos 0, 1.
 * The random streams are keyed by global cell numbers, so the strips
 * together follow the serial chain bit for bit.  Other entry points that
 * take an hdmc_t accept a strip handle only where noted (hdmc_sample,
 * hdmc_get_state (local rows, halos included), hdmc_counters (the strip's
 * own trials), hdmc_info, hdmc_sync, hdmc_set_stream, hdmc_set_move_size,
 * hdmc_set_balance, hdmc_destroy); the rest return HDMC_EINVAL. */

/* Creates strip `strip` (0 <= strip < nstrips) of the system hdmc_create
 * would build from the same arguments (hexagonal start), with device memory
 * from cudaMalloc, freed by hdmc_destroy.  Errors as hdmc_create, and
 * HDMC_EINVAL for a bad strip or my < 2 nstrips.  Synchronises. */
int hdmc_strip_create(hdmc_t **out, int64_t N, double Lx, double Ly, double sigma, double d, int nselect,
                      uint64_t seed, int precision, int32_t nstrips, int32_t strip, void *stream);

/* Global rows [first_row, end_row) the strip owns. */
int hdmc_strip_rows(hdmc_t *h, int32_t *first_row, int32_t *end_row);

/* Phase 1 of the next sweep: its draws and its four sub-sweeps (the band and
 * the halo rows make no moves).  Enqueued on the handle's stream.
 * HDMC_EINVAL if the previous sweep's shift is still missing. */
int hdmc_strip_subsweeps(hdmc_t *h);

/* Phase 2: the sweep's grid shift of the strip's own rows (Alg. 4); reads
 * the halo rows r_k - 1 and r_{k+1}.  HDMC_EINVAL without phase 1. */
int hdmc_strip_shift(hdmc_t *h);

/* Bytes of one cell row in the library's layout (mx cells, 8 coordinates
 * each: the even-x cells, then the odd-x cells). */
size_t hdmc_strip_row_bytes(const hdmc_t *h);

/* Copies an own row of the current state into buf (host or device memory,
 * hdmc_strip_row_bytes long): which = 0, 1, 2, 3 for rows r_k, r_k + 1,
 * r_{k+1} - 2, r_{k+1} - 1.  Synchronises the handle's stream. */
int hdmc_strip_get_row(hdmc_t *h, int32_t which, void *buf);

/* Replaces a halo row with buf (as written by hdmc_strip_get_row of the
 * strip that owns the row): which = 0, 1, 2, 3 for rows r_k - 2, r_k - 1,
 * r_{k+1}, r_{k+1} + 1.  Synchronises the handle's stream. */
int hdmc_strip_set_halo(hdmc_t *h, int32_t which, const void *buf);

/* The strip's contact histogram accumulated by hdmc_sample since the last
 * call (HDMC_HIST_BINS counts, host; ordered pairs with the first disk in
 * the strip's own rows) and the number of samples; clears it.  Synchronises. */
int hdmc_strip_histogram(hdmc_t *h, uint64_t *hist, int64_t *n_samples);

/* The Sec. 4 estimator on a histogram of n_samples configurations of N
 * disks in an Lx x Ly box (for example the sum of the strips' histograms):
 * g(R_i) (Eqs. gR, R), the degree-5 least-squares fit over (sigma, 1.02
 * sigma], g(sigma+) and beta P / rho = 1 + (pi/2) rho sigma^2 g(sigma+)
 * (Eq. P).  Host only. */
int hdmc_pressure_fit(const uint64_t *hist, int64_t n_samples, int64_t N, double Lx, double Ly, double sigma,
                      double *betaP_over_rho, double *g_contact);

/* ---- batched replicas ----------------------------------------------------
 * R independent systems advanced together: every stage of a sweep is one
 * launch over all replicas, recorded into CUDA graphs, so small systems share
 * the GPU instead of each launching its own kernels.  Replica r is exactly the
 * system hdmc_create(N[r], Lx[r], Ly[r], sigma, d[r], nselect[r], seeds[r],
 * precision, ...) would build and its trajectory is bit-identical to that
 * run (the random streams are keyed by the replica's seed); batching only
 * changes the launch layout. */
typedef struct hdmc_batch_handle hdmc_batch_t;

/* Device bytes for a batch (0 if a replica's parameters are invalid). */
size_t hdmc_batch_workspace_bytes(int R, const int64_t *N, const double *Lx, const double *Ly, double sigma,
                                  int precision);

/* Creates R replicas (1 <= R <= 65535); N, Lx, Ly, d, seeds: host arrays of
 * length R with the meaning of hdmc_create's arguments; nselect: host array
 * of length R or NULL (4 for every replica).  dev_workspace / stream as in
 * hdmc_create.  Errors as hdmc_create (the first failing replica decides).
 * Synchronises. */
int hdmc_batch_create(hdmc_batch_t **out, int R, const int64_t *N, const double *Lx, const double *Ly,
                      double sigma, const double *d, const int32_t *nselect, const uint64_t *seeds, int precision,
                      void *dev_workspace, size_t workspace_bytes, void *stream);

/* Enqueues n sweeps of every replica (Algorithm 1). */
int hdmc_batch_sweep(hdmc_batch_t *b, int64_t n);

/* Enqueues the contact histogram of every replica into its accumulator. */
int hdmc_batch_sample(hdmc_batch_t *b);

/* Per-replica pressure from the accumulated samples, as hdmc_pressure:
 * betaP_over_rho[R], g_contact[R], hist[R*HDMC_HIST_BINS] (each nullable).
 * Clears the accumulators.  Synchronises. */
int hdmc_batch_pressure(hdmc_batch_t *b, double *betaP_over_rho, double *g_contact, uint64_t *hist,
                        int64_t *n_samples);

/* Raw state of replica r in the layout of hdmc_get_state.  Synchronises. */
int hdmc_batch_get_state(hdmc_batch_t *b, int r, double *local, uint8_t *counts);

/* Replaces replica r's configuration, grid origin and sweep counter, as
 * hdmc_set_state does for a single system (same layout, same checks:
 * HDMC_EINVAL for a count above 4, a coordinate outside its cell or not a
 * binary32 value in a binary32 batch, or a disk total other than the
 * replica's N; nothing changes then).  The other replicas are untouched.
 * Synchronises. */
int hdmc_batch_set_state(hdmc_batch_t *b, int r, const double *local, const uint8_t *counts,
                         const double origin[2], uint64_t sweeps_done);

/* Batch snapshots, as hdmc_save / hdmc_load for every replica at once: a
 * 256-byte header (magic "HDMCBSN1", version, precision, R, sub-sweep
 * block height, sweeps, sample count), then at 256-byte aligned offsets one
 * record per replica (N, box, sigma, d, n_M, grid, seed, balance controls),
 * the replicas' device state words, their trial counter totals, their
 * histogram accumulators and the arena of cells.  Loading requires the same
 * replicas (N, box, sigma, grid) and precision; d, n_M, seeds, controls and
 * the block height come from the image.  The cells are checked on the
 * device, replica by replica, before anything is replaced; a bad image is
 * rejected with HDMC_EINVAL and the batch keeps its state.  Both
 * synchronise. */
size_t hdmc_batch_snapshot_bytes(const hdmc_batch_t *b);
int hdmc_batch_save(hdmc_batch_t *b, void *buf, size_t bytes);
int hdmc_batch_load(hdmc_batch_t *b, const void *buf, size_t bytes);

/* psi_6 of every replica, as hdmc_psi6 (no per-slot output): out[4r + k].
 * r_cut must suit every replica's cells.  Synchronises. */
int hdmc_batch_psi6(hdmc_batch_t *b, double r_cut, double *out);

/* Per-replica trial counters out[4r + k], k as in hdmc_counters.  Synchronises. */
int hdmc_batch_counters(hdmc_batch_t *b, uint64_t *out);

/* Geometry of replica r, sweeps done, its grid origin (nullable outputs). */
int hdmc_batch_info(hdmc_batch_t *b, int r, int32_t *mx, int32_t *my, double *wx, double *wy,
                    uint64_t *sweeps_done, double origin[2]);

/* Sets n_M of every replica (host array of R values in 1..255). */
int hdmc_batch_set_nselect(hdmc_batch_t *b, const int32_t *nselect);

/* Sets the sub-sweep block height (1, 2, 4 or 8 rows of 32 active cells;
 * binary32 batches only).  Results do not depend on it.  Synchronises. */
int hdmc_batch_set_rows(hdmc_batch_t *b, int32_t rows_per_block);

/* Per-replica balance controls, as hdmc_set_balance: shuffle_particles[R],
 * shuffle_sets[R] (host).  Synchronises. */
int hdmc_batch_set_balance(hdmc_batch_t *b, const int32_t *shuffle_particles, const int32_t *shuffle_sets);

/* Current launch configuration: cells per block row count of the sub-sweep
 * (block = 32 x rows active cells) and n_M of every replica (nselect[R]). */
int hdmc_batch_config(hdmc_batch_t *b, int32_t *rows_per_block, int32_t *nselect);

/* Autotuner (runs real sweeps, which advance every replica): picks the
 * sub-sweep block height among 32x1, 32x2, 32x4, 32x8 active cells by the
 * time of `sweeps` recorded sweeps (binary32 batches), then n_M in
 * {1, 2, 4, 8} (the same for every replica) maximising the net squared
 * displacement per disk and second over `sweeps` sweeps, summed over
 * replicas -- each disk's displacement is taken over its cell update, so
 * confinement to the cell counts against a large n_M (the paper tunes n_M
 * by an autocorrelation time per wall-clock second, Sec. 3.3).
 * 1 <= sweeps <= 4096.  Synchronises. */
int hdmc_batch_autotune(hdmc_batch_t *b, int64_t sweeps, int32_t *rows_per_block, int32_t *nselect_chosen);

/* Frees the batch (and the workspace if the library allocated it). */
void hdmc_batch_destroy(hdmc_batch_t *b);

/* Contact histogram for callers that cannot allocate device memory.  The
 * paper has no counterpart: this entry point exists for code that may not
 * call cudaMalloc (inside another framework's memory pool, a memory-capped
 * process, or a plugin that owns no GPU allocations).  It allocates nothing:
 * its only device scratch is a file-scope array of HDMC_NOALLOC_MAX_BINS
 * 64-bit counters that every GPU which loads the library keeps until the
 * process exits.
 *   dev_local: device, caller-owned, 16-byte aligned, 8*mx*my doubles in
 *              the layout of hdmc_get_state (slot j of canonical cell
 *              c = cy*mx + cx at [(4c+j)*2], [(4c+j)*2+1], cell-local
 *              coordinates; a slot is empty iff its x is negative, whatever
 *              the negative value).  Read only.
 *   mx, my:    cell grid (>= 4 each); wx, wy: cell widths used to translate
 *              neighbouring cells (pass the binary32 widths, widened, for a
 *              state of an HDMC_FP32_LOCAL system).
 *   sigma, nbins, dr: ordered pairs at distance r in [sigma, sigma + nbins dr)
 *              are counted in bins [sigma + b dr, sigma + (b+1) dr), decided
 *              on the binary64 r^2 against the squared bin edges, as
 *              hdmc_pressure does; 1 <= nbins <= HDMC_NOALLOC_MAX_BINS and
 *              sigma + nbins dr <= 2 min(wx, wy).
 *   hist:      host, nbins counts (output).
 *   stream:    cudaStream_t or NULL (legacy default stream).
 * Errors: HDMC_EINVAL for a size above the maximum, a dev_local that is
 * not 16-byte aligned or other invalid arguments (nothing is launched),
 * HDMC_ECUDA.  Synchronises the stream.
 * The first call on each device looks up the device address of the scratch
 * array (with that device current) and keeps it for the life of the
 * process.  cudaDeviceReset may move the array, so do not use this entry point in a
 * process that resets a device it has called it on.  All calls share the
 * array and each call clears it first, so calls that overlap on the GPU
 * (several streams or host threads) race. */
#define HDMC_NOALLOC_MAX_BINS 1024
int hdmc_histogram_noalloc(const double *dev_local, int32_t mx, int32_t my, double wx, double wy, double sigma,
                           int32_t nbins, double dr, uint64_t *hist, void *stream);

/* ---- three dimensions: hard spheres ----------------------------------------
 * The same method for N hard spheres of diameter sigma in a periodic
 * Lx x Ly x Lz box (the paper gives the 3-d case in words: eight
 * checkerboard sets, eight sub-sweeps per sweep, Sec. 2.1, 2.2 and 6):
 *   - cells: m_a = largest even integer <= L_a/sigma per axis (>= 4), widths
 *     w_a = L_a/m_a with wx^2 + wy^2 + wz^2 < 4 sigma^2, so that a cell holds
 *     at most HDMC3_SLOTS = 8 centres (each of its eight half-size boxes is
 *     less than sigma across); mx*my*mz < 2^32;
 *   - set Q = (cx mod 2) + 2 (cy mod 2) + 4 (cz mod 2); a sweep draws the
 *     order of the eight sets (Fisher-Yates) and a shift direction among
 *     +-x, +-y, +-z with a distance uniform in [0, w/2);
 *   - a cell update shuffles its spheres and makes n_M trial moves, each a
 *     displacement uniform in the ball of radius d, rejected when it leaves
 *     the cell or overlaps a sphere of the 27-cell neighbourhood;
 *   - pressure from the contact value, beta P / rho = 1 + (2 pi/3) rho
 *     sigma^3 g(sigma+), g(R_i) from spherical shells.
 * Conventions (return codes, host pointers, stream, synchronisation) are
 * those of the two-dimensional entry points above.  Canonical layout: cell
 * c = (cz*my + cy)*mx + cx, slot j, coordinate a (0 x, 1 y, 2 z) of a sphere
 * at local[(8c+j)*3 + a], relative to the cell's lower corner, in [0, w_a);
 * slot j is used iff j < counts[c]; unused slots read HDMC_EMPTY_SLOT. */
typedef struct hdmc3_handle hdmc3_t;
#define HDMC3_SLOTS 8

/* Creates a system.  xyz: NULL for the face-centred cubic start (N = 4 q^3;
 * site p = 4((k q + j) q + i) + s at ((b + s + 1/4) L_a/q) for unit cell
 * b = (i,j,k) and basis vector s in {(0,0,0), (1/2,1/2,0), (1/2,0,1/2),
 * (0,1/2,1/2)}, displaced uniformly within 0.01 sigma), else host global
 * coordinates xyz[3i + a] in [0, L_a] (slot order = order of i within a
 * cell).  d: maximum displacement, 0 < d < min(w)/2; nselect: n_M, 1..255;
 * precision: HDMC_FP64 or HDMC_FP32_LOCAL (binary32 cell-local offsets).
 * stream: cudaStream_t or NULL.  Device memory (two copies of the cells,
 * 8 slots x 3 coordinates per cell, plus a few kilobytes) is allocated with
 * cudaMalloc and freed by hdmc3_destroy.  Errors: HDMC_EINVAL, HDMC_EOVERLAP,
 * HDMC_EOVERFLOW, HDMC_ENOMEM, HDMC_ECUDA; *out is NULL on failure.
 * Synchronises. */
int hdmc3_create(hdmc3_t **out, int64_t N, double Lx, double Ly, double Lz, double sigma, double d,
                 int nselect, uint64_t seed, int precision, const double *xyz, void *stream);

/* Enqueues n sweeps: one launch of the sweep draws per 64 sweeps, then per
 * sweep eight sub-sweep launches and one cell-shift launch. */
int hdmc3_sweep(hdmc3_t *h, int64_t n);

/* Enqueues one extra cell shift drawn from the stream of explicit shifts. */
int hdmc3_shift(hdmc3_t *h);

/* Enqueues one sub-sweep of set Q (0..7) with the cell streams of sweep
 * index `sweep` (a test hook: a sweep is eight of these and a shift). */
int hdmc3_subsweep(hdmc3_t *h, uint32_t sweep, int Q);

/* Enqueues the contact histogram (ordered pairs at distance in
 * [sigma, 1.02 sigma), bins of 1e-4 sigma, decided in binary64 over the
 * 5x5x5 cell neighbourhood) and adds it to the sample accumulator. */
int hdmc3_sample(hdmc3_t *h);

/* Pressure from the accumulated samples (one sample of the current
 * configuration first if there is none): g(R_i) = n_i / (n_conf N rho
 * (4 pi/3)(r_{i+1}^3 - r_i^3)) at R_i = (3/4)(r_{i+1}^4 - r_i^4) /
 * (r_{i+1}^3 - r_i^3), the degree-5 least-squares polynomial over
 * (sigma, 1.02 sigma] evaluated at sigma, beta P / rho = 1 + (2 pi/3) rho
 * sigma^3 g(sigma+).  Outputs nullable as in hdmc_pressure.  Clears the
 * accumulator.  Synchronises. */
int hdmc3_pressure(hdmc3_t *h, double *betaP_over_rho, double *g_contact, uint64_t *hist, int64_t *n_samples);

/* Global coordinates into host xyz[3N] in canonical (cell, slot) order:
 * O_a + (c_a w_a + local_a) wrapped into [0, m_a w_a) (binary32 widths in
 * HDMC_FP32_LOCAL mode).  Synchronises. */
int hdmc3_positions(hdmc3_t *h, double *xyz);

/* Raw state in the canonical layout: local (host, 24 C doubles), counts
 * (host, C bytes), C = mx*my*mz.  Synchronises. */
int hdmc3_get_state(hdmc3_t *h, double *local, uint8_t *counts);

/* Cumulative trial counters as hdmc_counters.  Synchronises. */
int hdmc3_counters(hdmc3_t *h, uint64_t out[4]);

/* Grid m[3], widths w[3] (binary64), origin[3], sweeps and explicit shifts
 * done (each nullable).  Synchronises. */
int hdmc3_info(hdmc3_t *h, int32_t m[3], double w[3], double origin[3], uint64_t *sweeps_done,
               uint64_t *shifts_done);

/* Maximum displacement for the sweeps enqueued after the call
 * (0 < d < min(w)/2). */
int hdmc3_set_move_size(hdmc3_t *h, double d);

/* Balance controls as hdmc_set_balance (shuffle_sets = 0 takes the sets in
 * the order 0..7). */
int hdmc3_set_balance(hdmc3_t *h, int shuffle_particles, int shuffle_sets);

/* Snapshots of a sphere system, as hdmc_snapshot_bytes / hdmc_save /
 * hdmc_load for disks: a 256-byte header (magic "HDMC3SN1", format version,
 * precision, N, box, sigma, d, n_M, grid, seed, balance controls, sweep and
 * shift counters, accumulated sample count), then at 256-byte aligned
 * offsets the device state (trial counters, grid origin, error word), the
 * histogram accumulator and the cells in the device layout (primary halves
 * of all cells, then secondary halves; binary32 or binary64).  Load requires
 * the same N, box, sigma and precision, takes d, n_M, seed and the balance
 * controls from the image, and checks the cells on the device before
 * anything is replaced: a wrong header, an occupied slot after an empty one,
 * a coordinate outside [0, w), an empty slot not holding HDMC_EMPTY_SLOT in
 * all three coordinates, or a sphere total other than N gives HDMC_EINVAL
 * and the handle keeps its state.  Save and load synchronise. */
size_t hdmc3_snapshot_bytes(const hdmc3_t *h);
int hdmc3_save(hdmc3_t *h, void *buf, size_t bytes);
int hdmc3_load(hdmc3_t *h, const void *buf, size_t bytes);

/* Waits for the handle's stream and reports device-side errors. */
int hdmc3_sync(hdmc3_t *h);

/* Profiling form of hdmc3_sweep: n sweeps with the same results, an event
 * pair around every launch; mean milliseconds of one sub-sweep launch and
 * one shift launch (nullable).  Synchronises. */
int hdmc3_profile_sweeps(hdmc3_t *h, int64_t n, double *ms_subsweep, double *ms_shift);

/* In-step timing of the three-dimensional sweep, as hdmc_profile_stages:
 * n sweeps of the draws and eight sub-sweeps without shifts, then n sweeps of
 * the draws and the shift, each run timed as a whole with CUDA events on the
 * handle's stream; mean milliseconds per sub-sweep and per shift launch
 * (each nullable).  The configuration stays legal, the trajectory is not
 * that of hdmc3_sweep.  n >= 1.  Synchronises. */
int hdmc3_profile_stages(hdmc3_t *h, int64_t n, double *ms_subsweep, double *ms_shift);

/* Frees the handle. */
void hdmc3_destroy(hdmc3_t *h);

/* Frees the handle (and the workspace if the library allocated it). */
void hdmc_destroy(hdmc_t *h);

/* Static description of an error code. */
const char *hdmc_strerror(int code);

/* Build options of this libhdmc.so: HDMC_BUILD_CHECK when it was compiled
 * with -DHDMC_CHECK.  Such a build checks every cell index its kernels
 * compute against the grid; a bad index is replaced by 0 (so no access
 * leaves the buffer) and sets a bit of the handle's device error word, which
 * the next synchronising call reports as HDMC_ECHECK.  compute-sanitizer is
 * not available on every machine; this is its substitute for the kernels'
 * own index arithmetic.  Normal builds contain none of these checks. */
#define HDMC_BUILD_CHECK 1
int hdmc_build_flags(void);

#ifdef __cplusplus
}
#endif

#endif /* HDMC_H */
