/*
 * amber.h -- C ABI of libamber: the reionization-redshift assignment z_re(x)
 * of AMBER (Trac et al., arXiv 2109.10375) on one NVIDIA GB300 (sm_103a).
 *
 * The path, in the paper's order:
 *   amber_radiation_field  J = S * exp(-r/l_mfp)/(4 pi r^2) by FFT   (Sec. 3.4.1, Eq. intensity)
 *   amber_rank             order cells by J, descending               (Sec. 3.4.2)
 *   amber_assign_zre       cumulative-mass abundance matching to the
 *                          Weibull history x(z) of (z_mid, dz, Az)    (Sec. 3.4.2, Sec. 3.1, App. A)
 *   amber_solve            all of the above in one call
 *
 * Conventions for every entry point:
 *  - Fields are C-order [z][y][x] (x fastest) on a periodic n^3 grid of side
 *    `box` (h^-1 Mpc); n is a power of two in [4, 1024].
 *  - Pointers named d_* are DEVICE pointers owned by the caller (any CUDA
 *    allocation on the context's device).  The library never frees them.
 *    Each must start on a multiple of its element size (4 bytes for float
 *    and uint32 arrays, 8 for double); a misaligned pointer returns
 *    AMBER_ERR_INVALID_ARG with nothing enqueued.  No wider alignment is
 *    needed: an array may start anywhere on its element size (a view
 *    such as J + 1 is fine).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  All device work is asynchronous on that stream; no call
 *    allocates device memory after amber_create (amber_batch_create
 *    allocates its batch's own workspace).
 *  - Return values are amber_status codes.  Argument errors are detected on
 *    the host and returned immediately with nothing enqueued.  Errors found by
 *    kernels (non-finite intensity, invalid mass, a lookback wait that ran
 *    out) latch in a device status word read by amber_sync_status.
 *  - A context serialises its own work: calls on one context must not
 *    overlap in time on different streams (they share one workspace).
 *    Use one context per concurrent stream.
 */
#ifndef AMBER_H_
#define AMBER_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMBER_OK = 0,
  AMBER_ERR_INVALID_ARG = 1,     /* bad size, pointer, box, l_mfp or history point */
  AMBER_ERR_NO_SOLUTION = 2,     /* no Weibull root with a_w, b_w, c_w > 0 (App. A) */
  AMBER_ERR_NONFINITE = 4,       /* device: a NaN or Inf intensity was ranked */
  AMBER_ERR_OOM = 8,             /* workspace allocation failed in amber_create */
  AMBER_ERR_DEVICE_TIMEOUT = 16, /* device: a bounded lookback wait ran out */
  AMBER_ERR_CUDA = 32,           /* a CUDA runtime call failed (no device, launch error) */
  AMBER_ERR_INVALID_MASS = 64,   /* device: a cell mass was negative, NaN or >= 2^40 */
  AMBER_ERR_CAPACITY = 128       /* size exceeds the context's max_cells */
} amber_status;

typedef struct amber_ctx amber_ctx;

/* Weighting of the cumulative ionized fraction that abundance matching
 * equates with the history x(z) (Sec. 3.4.2):
 *   AMBER_WEIGHT_MASS         cell weight = its mass, the same at every z (the
 *                             plain path: no growth rescaling);
 *   AMBER_WEIGHT_MASS_GROWTH  cell weight at redshift z = 1 + delta_m(z) with
 *                             delta_m(z) = D(z)/D(z_mid) delta_m(z_mid) and
 *                             delta_m(z_mid) = mass - 1 (the mass field read as
 *                             1 + delta at the midpoint), D the linear growth
 *                             factor of flat LCDM with Omega_m = omega_m (the
 *                             full equation of Sec. 3.4.2);
 *   AMBER_WEIGHT_VOLUME       every cell weighs 1 (the volume-weighted fraction,
 *                             Sec. 2.3 and 3.1.1). */
enum { AMBER_WEIGHT_MASS = 0, AMBER_WEIGHT_MASS_GROWTH = 1, AMBER_WEIGHT_VOLUME = 2 };

/* Reionization history (Sec. 3.1.1): midpoint, duration dz = z_ear - z_lat,
 * asymmetry Az = (z_ear - z_mid)/(z_mid - z_lat); the ionized fractions at
 * the three points (default 0.05, 0.50, 0.95); the table x(z_j) on n_table
 * uniform redshifts in [min(z_lo, a_w), z_hi] (default 5, 20, 2000); and the
 * weighting of the matched fraction (default AMBER_WEIGHT_MASS) with the
 * matter density parameter its growth factor uses (default 0.3, Sec. 2). */
typedef struct {
  double z_mid, dz, Az;
  double x_ear, x_mid, x_lat;
  double z_lo, z_hi;
  int n_table;
  int weighting;
  double omega_m;
} amber_history_t;

/* One realisation's parameters.  precision: 32 (FP32 FFT and intensity) or
 * 64 (FP64 FFT and intensity, n <= 256). */
typedef struct {
  int n;
  double box;
  double l_mfp;
  amber_history_t hist;
  int precision;
} amber_params_t;

/* Fill *h with the paper's defaults (x points 0.05/0.50/0.95, table [5,20] x 2000,
 * mass weighting, Omega_m 0.3). */
int amber_history_default(amber_history_t *h, double z_mid, double dz, double Az);

/* Weibull coefficients (a_w, b_w, c_w) of x(z) = exp(-max((z-a)/b,0)^c) through
 * the three ionization points (Sec. 3.1.2, Eq. weibull; App. A).  Host only, FP64,
 * no GPU needed.  The root in c is bracketed on a log grid over [0.05, 100] and
 * bisected (the appendix's secant iteration can leave the valid region).
 * z_lat is taken as z_ear - dz (the duration definition).
 * Returns AMBER_ERR_INVALID_ARG for points not 0 < x_ear < x_mid < x_lat < 1,
 * dz <= 0 or Az <= 0; AMBER_ERR_NO_SOLUTION if no positive root exists. */
int amber_history_coeffs(const amber_history_t *h, double out_abc[3]);

/* The history table the device builds for h, computed on the host in FP64:
 * z_out[j], x_out[j] for j < h->n_table (caller-owned host arrays).  Host only. */
int amber_history_table(const amber_history_t *h, double *z_out, double *x_out);

/* Create a context on `device` able to process up to max_cells cells
 * (max_cells <= 2^30; the FFT needs n^3 <= max_cells).  Allocates the whole
 * workspace once (about 29 bytes per cell including the half spectrum, see
 * amber_workspace_bytes).  *ctx is owned by the caller and released with
 * amber_destroy.  Returns AMBER_ERR_CUDA when no device is usable and
 * AMBER_ERR_OOM when the workspace does not fit. */
int amber_create(amber_ctx **ctx, int device, int64_t max_cells);
int amber_destroy(amber_ctx *ctx);

/* Bytes of device workspace amber_create(max_cells) allocates.  Host only. */
int amber_workspace_bytes(int64_t max_cells, size_t *out_bytes);

/* Radiation intensity (Sec. 3.4.1, Eq. intensity):
 *   J = IDFT( DFT(S) * arctan(|k| l_mfp)/|k| ),  value l_mfp at k = 0,
 * the periodic convolution of S with exp(-r/l_mfp)/(4 pi r^2), where
 * k = 2 pi m / box for signed FFT index m and the inverse carries 1/n^3.
 * d_src: n^3 floats (cell order); d_J: n^3 floats out (may alias d_src).
 * FP32 arithmetic, twiddles rounded from FP64. */
int amber_radiation_field(amber_ctx *ctx, const float *d_src, int n, double box, double l_mfp,
                          float *d_J, void *stream);
/* Same in FP64 (n <= 256): d_src and d_J are n^3 doubles. */
int amber_radiation_field_f64(amber_ctx *ctx, const double *d_src, int n, double box, double l_mfp,
                              double *d_J, void *stream);

/* Ranking (Sec. 3.4.2): d_order[r] = index of the cell with rank r, ranks in
 * descending J, equal J ordered by ascending cell index (a stable sort; the
 * paper's quicksort leaves ties unspecified).  -0.0 ranks equal to +0.0.
 * A NaN intensity latches AMBER_ERR_NONFINITE.  ncells in [1, max_cells].
 * d_J: ncells floats; d_order: ncells uint32 out. */
int amber_rank(amber_ctx *ctx, const float *d_J, int64_t ncells, uint32_t *d_order, void *stream);
/* Same for FP64 intensities (ncells <= 2^24). */
int amber_rank_f64(amber_ctx *ctx, const double *d_J, int64_t ncells, uint32_t *d_order, void *stream);

/* Abundance matching (Sec. 3.4.2): with M_n = sum_{m<=n} mass[order[m]] and
 * F_n = M_n / M_{ncells-1}, the rank-n cell gets z_n from the tabulated
 * history: j* = largest j with x(z_j) >= F_n; z_n = z_lo if there is none,
 * z_hi if j* is the last node, otherwise the linear interpolation
 * z_j* + (x_j* - F_n)/(x_j* - x_j*+1) (z_j*+1 - z_j*).  Writes
 * d_zre[order[n]] = z_n (float, cell order).
 * The mass total is exact (128-bit fixed point, 2^-64 units); the running
 * prefix M_n is 64-bit fixed point with a shift s chosen from the total so
 * it stays below 2^62 (each mass rounded down to a multiple of 2^-s), so F_n
 * is within n 2^-60 of the exact value; the bracket test "x_j >= F_n" is an
 * exact integer comparison against thresholds floor(x_j T) in the same fixed
 * point, and only the interpolation weight is FP32.  No result depends on
 * the order of addition.  d_F_opt, if not NULL, receives F_n (double, rank
 * order).
 * Masses must be finite, >= 0 and < 2^40 (else AMBER_ERR_INVALID_MASS latches),
 * with a total in (0, 2^63).  d_order must be a permutation of [0, ncells).
 *
 * Other weightings (h->weighting, see AMBER_WEIGHT_*): the weight of cell m
 * at table redshift z_j is alpha_j + beta_j mass_m, so its cumulative sum is
 * W_n(z_j) = alpha_j n + beta_j M_n with n counting ranks from 1.  The rank-n
 * cell is ionized at z_j when W_n(z_j) <= x_j W_N(z_j); its redshift comes
 * from the largest such j, call it k (the cell's first ionization: with
 * grown weights that turn negative in deep voids the fraction can cross x(z)
 * more than once), interpolated linearly where the margin
 * h_j = x_j W_N(z_j) - W_n(z_j) changes sign: t = h_k / (h_k - h_k+1),
 * z_n = z_k + t (z_k+1 - z_k).  The mass weighting reduces to the rule above.  These margins are evaluated in FP32 (about 1e-7 of W_N), and
 * d_F_opt still receives the mass fraction M_n / M_total. */
int amber_assign_zre(amber_ctx *ctx, const uint32_t *d_order, const float *d_mass, int64_t ncells,
                     const amber_history_t *h, float *d_zre, double *d_F_opt, void *stream);

/* Source field from a density field (the step before the radiation field in
 * the serving path).  Sec. 3.3's excursion-set collapsed fraction with the
 * ESF-E halo density (Eq. fcoll; rho_h = f_coll rho (1 + delta)):
 *   mass = 1 + max(delta, -0.99),
 *   S = mass * erfc((delta_c - delta)/(sqrt(2) sigma_f)), then S /= mean(S),
 * with sigma_f standing in for sqrt(sigma^2(M_min) - sigma^2(M_s)).
 * d_delta: ncells floats; d_S: ncells floats out; d_mass_opt: ncells floats
 * out or NULL.  FP32 elementwise, exact fixed-point mean.  A NaN density
 * latches AMBER_ERR_NONFINITE. */
int amber_source_field(amber_ctx *ctx, const float *d_delta, int64_t ncells, double delta_c, double sigma_f,
                       float *d_S, float *d_mass_opt, void *stream);

/* The whole path for one realisation: radiation field -> rank -> assign.
 * d_src, d_mass: n^3 floats; d_zre: n^3 floats out; d_J_opt: if not NULL,
 * n^3 floats out with the intensity.  p->precision must be 32 here. */
int amber_solve(amber_ctx *ctx, const float *d_src, const float *d_mass, const amber_params_t *p,
                float *d_zre, float *d_J_opt, void *stream);
/* amber_solve from and to HOST memory: h_src and h_mass (n^3 floats each,
 * host) are copied to the device, solved as by amber_solve, and z_re (n^3
 * floats) copied back to h_zre, all in order on `stream`; the call returns
 * once the work is enqueued, and h_zre holds the result after the stream has
 * reached it (synchronise the stream or an event).  Host buffers allocated
 * pinned (cudaMallocHost, cudaHostRegister) copy at the link's full rate and
 * asynchronously; pageable ones are copied through the driver's staging.
 * No device memory beyond the context's workspace: the copies live in
 * workspace that is free while they are needed.  To overlap one step's
 * copies with another's solve, alternate two or more contexts, each on its
 * own stream: host-buffer solves on one device take turns in call order (a
 * call's solve waits for the previous call's solve, on whichever context, but
 * its copies in do not), so the copies of one call run while another solves
 * and no two of these solves share the GPU. */
int amber_solve_host(amber_ctx *ctx, const float *h_src, const float *h_mass, const amber_params_t *p,
                     float *h_zre, void *stream);

/* amber_solve that also hands back what a parameter study reuses: the rank
 * order (d_order_out, n^3 uint32) and the masses in rank order
 * (d_mass_rank_out, n^3 floats), both caller-owned device buffers.  A later
 * change of only (z_mid, dz, Az) reruns amber_assign_zre_ranked on them. */
int amber_solve_ex(amber_ctx *ctx, const float *d_src, const float *d_mass, const amber_params_t *p,
                   float *d_zre, float *d_J_opt, uint32_t *d_order_out, float *d_mass_rank_out, void *stream);

/* amber_assign_zre with the masses already in rank order (d_mass_rank[n]
 * belongs to the cell d_order[n]), as amber_solve_ex leaves them: the same
 * abundance matching without the gather through the order. */
int amber_assign_zre_ranked(amber_ctx *ctx, const uint32_t *d_order, const float *d_mass_rank, int64_t ncells,
                            const amber_history_t *h, float *d_zre, double *d_F_opt, void *stream);

/* ---- Reuse of the transformed source field (parameter studies) --------- */

/* Bytes of the transformed source field of an n^3 grid that
 * amber_source_spectrum writes: n^2 (n/2 + 2) complex64 values.  Host only. */
int amber_spectrum_bytes(int n, size_t *out_bytes);

/* The first two of the radiation field's five passes (Sec. 3.4.1): the
 * real-to-complex transform along x and the forward transform along y of
 * the source d_src (n^3 floats), written to d_spec (caller-owned device
 * memory of amber_spectrum_bytes(n) bytes, 16-byte aligned; layout
 * [z][y][kx] complex64, kx in [0, n/2] on rows of n/2 + 2).  The z transform
 * is left to amber_solve_spectrum, which fuses it with the kernel multiply,
 * so a parameter study that varies l_mfp (Sec. 5) keeps d_spec per source
 * field and skips these passes.  Uses the context's FFT tile variant for n
 * (amber_tuning_t). */
int amber_source_spectrum(amber_ctx *ctx, const float *d_src, int n, void *d_spec, void *stream);

/* amber_solve_ex starting from d_spec (amber_source_spectrum's output, only
 * read): the forward z transform with the kernel multiply for p->l_mfp, the
 * inverse transforms, ranking and matching.  With the same context tuning
 * the results equal amber_solve_ex's on the source field bit for bit.
 * d_order_out and d_mass_rank_out are both given (as for amber_solve_ex)
 * or both NULL. */
int amber_solve_spectrum(amber_ctx *ctx, const void *d_spec, const float *d_mass, const amber_params_t *p,
                         float *d_zre, float *d_J_opt, uint32_t *d_order_out, float *d_mass_rank_out, void *stream);

/* ---- Autotuning of the FP32 solve path per grid size ------------------- */

/* The choices the FP32 solve path (amber_solve, amber_solve_ex,
 * amber_solve_tomographic, amber_batch_*) and the FP32 amber_radiation_field
 * make for one grid size n of one context:
 *   fft_variant      0: the default tiles (every n); 1: an alternative radix
 *                    split or tile width (n >= 128: 1024 with 4-line tiles,
 *                    512 as 16 x 32, 256 as 32 x 8, 128 as 8 x 16);
 *   sort_digit_bits  9 or 8: digit width of the radix sort (a few-octave
 *                    intensity field needs 27 bits: 3 passes of 9 bits, 4 of 8;
 *                    a 24-bit range takes 3 of either, the 8-bit ones cheaper);
 *   sort_match       0: digit peers by one warp ballot per digit bit;
 *                    1: by warp match (AMBER_SORT_RANK=ballot|match in the
 *                    environment overrides it);
 *   fuse_histogram   with 8-bit digits, 1: the solve's inverse x pass counts
 *                    the intensities' digits as it writes them and the sort
 *                    runs on the raw 32-bit keys (always four passes) with no
 *                    histogram pass of its own; 0: a histogram pass of
 *                    key - min(key) (a narrow key range may need fewer passes);
 *   zpass_tma        1: the fused z pass (n >= 64) is a persistent kernel whose
 *                    tiles arrive in shared memory by TMA (cp.async.bulk.tensor
 *                    under a 3D tensor map of the half spectrum), the next
 *                    tile's copy overlapping the current tile's stores;
 *                    0: each CTA loads its tile with ordinary loads.  The
 *                    arithmetic is the same, so are the results, bit for bit.
 * Every choice gives the same ranking (the stable descending order is
 * unique); the FFT variants differ only in FP32 rounding.  Defaults: 0, 8
 * for n >= 512 and 9 below, 0, 0 but 1 for n = 512 (the tuner's picks on a
 * synthetic field of the paper's kind).
 * tuned: 1 once amber_autotune measured this size; fft_ms[v] and sort_ms[k]
 * hold the median times it measured (k: (9, ballot), (9, match), (8,
 * ballot), (8, match); 0 where not applicable), fft_tma_ms the radiation
 * field's with the chosen variant and the TMA z pass (0 below n = 64). */
typedef struct {
  int n;
  int fft_variant;
  int sort_digit_bits;
  int sort_match;
  int tuned;
  double fft_ms[2];
  double sort_ms[4];
  int fuse_histogram;
  int zpass_tma;
  double fft_tma_ms;
} amber_tuning_t;

/* Measures every choice on the caller's own field (d_src, d_mass: n^3 floats
 * each, the solve's inputs; box and l_mfp as for amber_solve), keeps the
 * fastest for n on this context and writes the result to *out (may be NULL).
 * Each candidate runs once untimed and three times timed (CUDA events; the
 * median counts); the ranking is timed with the mass payload as in the
 * solve.  Synchronises the stream.  Leaves no result in the caller's
 * buffers; overwrites the context's workspace.  Errors as for amber_solve. */
int amber_autotune(amber_ctx *ctx, const float *d_src, const float *d_mass, int n, double box, double l_mfp,
                   amber_tuning_t *out, void *stream);
/* Sets the choices for t->n explicitly (t->tuned and the times are kept as
 * given).  AMBER_ERR_INVALID_ARG for a size the context cannot hold or a
 * choice out of range. */
int amber_set_tuning(amber_ctx *ctx, const amber_tuning_t *t);
/* The current choices for size n. */
int amber_get_tuning(amber_ctx *ctx, int n, amber_tuning_t *out);

/* Batched solves: many realisations of mixed grid sizes, every stage of
 * every item in one launch per stage, captured once into a CUDA graph.
 *  - The transforms run one launch per pass and grid size (the items of a
 *    size back to back), the ranking one histogram, one digit-offset and one
 *    launch per digit pass per digit width, the matching one thresholds, one
 *    scan per weighting form and one scatter launch for all items.  Inside a
 *    launch each CTA finds its item from a prefix of the items' tile counts;
 *    ticket-ordered kernels (digit passes, scan) take tiles from the item's
 *    own ticket, so their look-backs stay within the item.  The graph's
 *    kernel nodes number 5 per grid size plus 6 per digit width plus 3 or 4,
 *    whatever the item count (amber_batch_kernel_nodes).
 *  - The batch allocates its own workspace at creation (about 30 bytes per
 *    cell of all items together, plus the items' arguments); amber_batch_create
 *    and amber_create are the only calls that allocate.
 *  - ctxs[0] gives the device, the FFT twiddles (its max_cells must hold the
 *    largest grid), the status word that amber_sync_status(ctxs[0]) reads and
 *    the tuning; each grid size not yet tuned on ctxs[0] is autotuned on its
 *    first item (amber_autotune) unless AMBER_AUTOTUNE=0 is set, and the
 *    choices are copied to every context given.  Other contexts do no work.
 *  - Items are validated before anything runs (the rules of amber_solve,
 *    precision 32, and n >= 8).  Results equal amber_solve's on ctxs[0] with
 *    the same tuning, bit for bit.
 *  - The graph records the given device pointers and parameters: the items'
 *    buffers and ctxs[0] must stay alive while the batch exists, and ctxs[0]
 *    must not run other work while the batch runs. */
typedef struct {
  const float *d_src;
  const float *d_mass;
  amber_params_t params;
  float *d_zre;
} amber_batch_item;
typedef struct amber_batch amber_batch;
int amber_batch_create(amber_batch **batch, amber_ctx *const *ctxs, int nctx, const amber_batch_item *items,
                       int nitems);
int amber_batch_launch(amber_batch *batch, void *stream);
/* Kernel nodes in the batch's graph (host only). */
int amber_batch_kernel_nodes(amber_batch *batch, int *out_nodes);
int amber_batch_destroy(amber_batch *batch);

/* FP64 intensity variant (p->precision == 64, n <= 256): d_src n^3 doubles,
 * d_J_opt n^3 doubles or NULL. */
int amber_solve_f64(amber_ctx *ctx, const double *d_src, const float *d_mass, const amber_params_t *p,
                    float *d_zre, double *d_J_opt, void *stream);

/* Synchronise `stream`, return and clear the device status word (OR of
 * amber_status bits latched by kernels since the last call). */
int amber_sync_status(amber_ctx *ctx, void *stream);

/* Human-readable name of a status code (static string). */
const char *amber_status_string(int code);

/* The layout of a public struct as this library was compiled, so a binding
 * in another language can check its own copy: which = 0 amber_history_t,
 * 1 amber_params_t, 2 amber_tuning_t, 3 amber_batch_item.  Writes sizeof to
 * *size and the byte offset of each member, in declaration order, to
 * offsets[0 .. *count - 1] (at most max_offsets of them; *count is the
 * member count).  Host only: no CUDA call, no context.  AMBER_ERR_INVALID_ARG
 * for another `which` or a NULL size or count. */
int amber_struct_layout(int which, size_t *size, size_t *offsets, int max_offsets, int *count);

/* Per-kernel timing with CUDA events on the launching stream.  When enabled,
 * every kernel launch is bracketed by events and the totals accumulate until
 * amber_profile_reset.  amber_profile_read synchronises the context's last
 * stream and returns, for kernel kind `kind` (0 <= kind < amber_profile_kinds()),
 * its name, total milliseconds and launch count. */
int amber_profile_enable(amber_ctx *ctx, int on);
int amber_profile_reset(amber_ctx *ctx);
int amber_profile_kinds(void);
int amber_profile_read(amber_ctx *ctx, int kind, const char **name, double *total_ms, int64_t *launches);

/* Digit passes the last ranking needed (diagnostic; synchronises the
 * context's last stream).  The sort runs on key - min(key) with 9- or 8-bit
 * digits (amber_tuning_t), so an intensity field spanning few octaves (27
 * bits) needs 3 or 4 passes; at most 4 for FP32 keys. */
int amber_sort_passes(amber_ctx *ctx, int *out_passes);

/* Tomographic abundance matching (Sec. 3.4.2 names matching over several
 * redshift intervals as an option, without further detail).  Interval k = 0..nint-1
 * covers [z_bounds[k+1], z_bounds[k]) (host array, strictly decreasing, nint
 * in [1, 64]) and has its own source field d_src_list[k] (n^3 floats each,
 * e.g. the sources at the interval's redshift).  For each interval, from high
 * to low redshift: J_k = the radiation field of d_src_list[k]; cells that
 * already have a redshift rank first (they take the next float above the
 * largest J_k, and among themselves cell order: they hold the earliest share
 * of the ionized mass), the rest by descending J_k; abundance matching
 * over that ranking (the plain mass weighting of p->hist) gives each
 * still-neutral cell a redshift, which it keeps if it is at or above
 * z_bounds[k+1] (always, in the last interval).  With the same source in
 * every interval the result equals amber_solve's exactly (the prefix sums
 * are exact, so their order does not matter).  Costs one radiation field,
 * one ranking and one matching per interval.  d_zre: n^3 floats out. */
int amber_solve_tomographic(amber_ctx *ctx, const float *const *d_src_list, int nint, const double *z_bounds,
                            const float *d_mass, const amber_params_t *p, float *d_zre, void *stream);

/* ---- Source-field pipeline (Sec. 3.2, 3.2.1, 3.3) ----------------------- */

/* Second-order Lagrangian displacement (Sec. 3.2, Eq. xlpt) of one particle
 * per lattice point q of an n^3 periodic box of side `box`:
 *   psi = x - q = -D1 grad phi1 + D2 grad phi2,
 *   lap phi1 = delta_lin,  lap phi2 = sum_{i<j} [phi1,ii phi1,jj - (phi1,ij)^2],
 * derivatives spectral (phi at k = 0 is 0; an odd derivative along an axis
 * at its Nyquist wave number is 0).  D1, D2: the first- and second-order
 * growth factors at the target redshift (the usual D2 = -3/7 D1^2).
 * d_delta_lin: n^3 floats [z][y][x], the linear overdensity the growth
 * factors scale; d_psi_x/y/z: n^3 floats each out, box units (also used as
 * scratch).  FP32 transforms.  Uses the context's transform, sort and mass
 * buffers; n a power of two in [4, 1024] with n^3 <= max_cells. */
int amber_lpt_displacement(amber_ctx *ctx, const float *d_delta_lin, int n, double box, double D1, double D2,
                           float *d_psi_x, float *d_psi_y, float *d_psi_z, void *stream);

/* Mesh density rho / <rho> (Sec. 3.2.1) from particles at q + psi (one per
 * lattice point, periodic) with masses d_mass_opt (n^3 floats, NULL: all
 * equal), assigned to the mesh points x_n = n dx with the order-`order`
 * window: 1 NGP, 2 CIC, 3 TSC (particle at distance d in [-1/2, 1/2) cells
 * from its nearest mesh point).  interlace = 1: a second mesh whose particles
 * move by dx/2 on every axis, combined as [rho1(k) + e^{i k.dX} rho2(k)] / 2 /
 * W(k) with W the window's transform [prod sin(k_a dx/2)/(k_a dx/2)]^order
 * (Eqs. interlace, Wofk); modes with a Nyquist component are dropped (after
 * the half-cell twiddle they have no real counterpart).  interlace = 0: the
 * plain assignment, not deconvolved.  FP32 atomics (sums in any order).
 * d_rho: n^3 floats out. */
int amber_mesh_density(amber_ctx *ctx, const float *d_psi_x, const float *d_psi_y, const float *d_psi_z,
                       const float *d_mass_opt, int n, double box, int order, int interlace, float *d_rho,
                       void *stream);

/* ESF collapsed fraction (Sec. 3.3, Eq. fcoll): delta_f = delta_lin filtered
 * with a sharp k-space window (filter 0: W = 1 for k R <= 1, else 0) or a
 * spherical top hat (filter 1: W = 3 (sin x - x cos x)/x^3, x = k R), then
 * f_coll = erfc[(delta_c - delta_f) / sqrt(2 dsigma2)] with delta_c the
 * barrier delta_crit / D(z) and dsigma2 = sigma^2(M_min) - sigma^2(M_s).
 * In ESF-L the particles then carry f_coll m_p to amber_mesh_density.
 * d_fcoll: n^3 floats out. */
int amber_esf_fcoll(amber_ctx *ctx, const float *d_delta_lin, int n, double box, double R, int filter,
                    double delta_c, double dsigma2, float *d_fcoll, void *stream);

/* sigma^2(R) = int Delta^2_lin(k) |W_th(k R)|^2 dln k (Sec. 3.3, Eq. variance)
 * by the trapezoid rule over a tabulated dimensionless linear power spectrum
 * (k increasing and positive, nk >= 2).  Host only, FP64. */
int amber_sigma2_tophat(const double *k, const double *Delta2, int nk, double R, double *out);

/* ---- Analysis of z_re fields (Sec. 2.3) -------------------------------- */

/* Normalised redshift field (Eq. deltaz): d_out[x] = ((1 + z[x]) - (1 + zbar))
 * / (1 + zbar) with zbar the volume-weighted (cell) mean of d_z, summed in
 * FP64; the field itself is FP32.  d_z, d_out: ncells floats (may alias);
 * d_zbar_opt: one device double out, or NULL. */
int amber_delta_z(amber_ctx *ctx, const float *d_z, int64_t ncells, float *d_out, double *d_zbar_opt,
                  void *stream);

/* PDF of the fractional difference (Eq. epsz) eps = ((1 + z) - (1 + z_ref)) /
 * (1 + z_ref), FP32 per cell: d_counts[0] counts eps < lo (and NaN),
 * d_counts[1 + i] the bin [lo + i w, lo + (i+1) w), w = (hi - lo)/nbins, and
 * d_counts[nbins + 1] eps >= hi (nbins + 2 uint64, device, zeroed here).
 * d_moments_opt: two device doubles out, sum of eps and of eps^2 (FP64), for
 * the mean and rms width.  nbins in [1, 16000], lo < hi finite. */
int amber_epsilon_z_pdf(amber_ctx *ctx, const float *d_z, const float *d_zref, int64_t ncells, double lo,
                        double hi, int nbins, unsigned long long *d_counts, double *d_moments_opt, void *stream);

/* Number of spherical shells amber_power_spectrum returns for an n^3 grid:
 * round(sqrt(3) n / 2) + 1 (n a power of two in [4, 1024]).  Host only. */
int amber_power_bins(int n, int *nbins);

/* Auto and cross power spectra (Eqs. Pk, Dk) of real n^3 fields a and b on a
 * periodic box of side `box`: P_ij(k) = <delta_i(k) delta_j(k)*> over the
 * modes of each spherical shell, in the continuum normalisation
 * delta(k) = (box/n)^3 sum_x delta(x) e^{-i k.x}, P = |delta(k)|^2 / box^3.
 * Shell b holds every wave vector of the full n^3 transform with integer
 * components m in [-n/2, n/2) and round(|m|) = b (k = 2 pi m / box), decided
 * exactly in integers; modes of the half spectrum with 0 < kx < n/2 count
 * twice (their conjugates).  Outputs (device doubles, amber_power_bins(n)
 * each, caller-owned): d_k mean |k| of the shell's modes, d_Paa, d_Pbb_opt,
 * d_Pab_opt (Re P_ab; zero without b), d_modes the number of modes.  With
 * these, Delta^2 = k^3 P / (2 pi^2), b_ab = sqrt(P_aa / P_bb) and
 * r_ab = P_ab / sqrt(P_aa P_bb) (Eqs. bias, rcc).  FP32 transforms, FP64 shell
 * sums.  d_b_opt may be NULL (auto spectrum of a only).  amber_power_derived
 * forms Delta^2, b and r on the device.  Uses the context's
 * transform and sort buffers; n^3 <= max_cells (else AMBER_ERR_CAPACITY). */
int amber_power_spectrum(amber_ctx *ctx, const float *d_a, const float *d_b_opt, int n, double box, double *d_k,
                         double *d_Paa, double *d_Pbb_opt, double *d_Pab_opt, double *d_modes, void *stream);

/* Statistics derived from amber_power_spectrum's shell averages, FP64 on the
 * device, per shell b < nbins (Sec. 2.3.1):
 *   d_D2aa[b] = k^3 P_aa / (2 pi^2)           (Eq. Dk; d_D2bb_opt likewise for b)
 *   d_bias_opt[b] = sqrt(P_aa / P_bb)          (Eq. bias)
 *   d_r_opt[b] = P_ab / sqrt(P_aa P_bb)        (Eq. rcc)
 * Inputs d_k, d_Paa, d_Pbb_opt, d_Pab_opt and outputs are device arrays of
 * nbins doubles (caller-owned; amber_power_bins gives nbins).  The outputs
 * for b need d_Pbb_opt, and d_r_opt needs d_Pab_opt too (else
 * AMBER_ERR_INVALID_ARG).  A shell without modes (P = 0) gets Delta^2 = 0
 * and NaN ratios. */
int amber_power_derived(amber_ctx *ctx, const double *d_k, const double *d_Paa, const double *d_Pbb_opt,
                        const double *d_Pab_opt, int nbins, double *d_D2aa, double *d_D2bb_opt, double *d_bias_opt,
                        double *d_r_opt, void *stream);

/* Test hook for failure detection: runs the production lookback wait on a
 * status array nothing ever publishes, with `spin_limit` iterations, and
 * latches AMBER_ERR_DEVICE_TIMEOUT.  No fault, no trap: the kernel returns. */
int amber_test_wait_timeout(amber_ctx *ctx, unsigned int spin_limit, void *stream);

/* Ranking without any device allocation, for callers that cannot allocate:
 * a plug-in inside a framework that owns the whole device pool, a real-time
 * loop that must never reach cudaMalloc (it can synchronise the device), or a
 * process whose memory is already handed out.  The paper has no counterpart;
 * this is an operational variant of amber_rank (same result, same order,
 * same tie rule) that needs no context.
 *  - Scratch: one fixed array of about 17 MB compiled into the library and
 *    held on every GPU that loads it until the process exits; it fits
 *    ncells <= 2^20.  Larger ncells return AMBER_ERR_CAPACITY and enqueue
 *    nothing.
 *  - The first call on each device (that device current) looks up the
 *    array's device address; make that first call before any stream capture.
 *    The address is kept for the life of the process, so this entry point is
 *    not valid after a cudaDeviceReset (or any teardown of the device's
 *    primary context) in the same process.
 *  - Every call shares the one array and clears what must start at zero; calls
 *    whose GPU work overlaps (other streams, other threads) race and must not
 *    be issued.  Runs on the current device, asynchronously on `stream`.
 *  - d_J: ncells floats; d_order: ncells uint32 out (caller-owned device
 *    memory); d_status_opt: a caller-owned device word into which device errors
 *    (AMBER_ERR_NONFINITE, AMBER_ERR_DEVICE_TIMEOUT) are ORed, or NULL to
 *    drop them.  No cudaMalloc, cudaFree or allocating library call. */
int amber_rank_noalloc(const float *d_J, int64_t ncells, uint32_t *d_order, unsigned int *d_status_opt,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* AMBER_H_ */
