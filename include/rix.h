/*
 * rix.h: C ABI of the GB300 (sm_103a) implementation of the per-partition
 * major-cycle measurement operator and minor cycles of the decentralized
 * radio-interferometric reconstruction of arXiv 2507.22128 ("A Decentralized
 * Framework for Radio-Interferometric Image Reconstruction").
 *
 * Conventions shared by every call
 * --------------------------------
 * Image: N x N, row-major, row b <-> direction cosine m = (b - N/2) dl, column
 *   a <-> l = (a - N/2) dl (phase centre at pixel (N/2, N/2)).  Real-valued,
 *   float (RIX_FP32 jobs) or double (RIX_FP64 jobs).
 * Visibilities: sample s = row * nchan + chan, complex interleaved
 *   (float2 / double2), layout [nrow][nchan].
 * uvw: float64 [nrow][3] in metres; u_lambda = u_m * f_chan / c.
 * Weights: float32 [nrow][nchan]; NULL means natural weights of 1.
 * Measurement model (Eq. 1, C = D = 1): V = sum I / n exp(-2 pi i (u l + v m +
 *   w (n - 1))), with the w-term and 1/n dropped in coplanar jobs
 *   (n_wplanes = 0).  Gridding: exponential-of-semicircle kernel, support 8,
 *   beta = 18.4, oversampling 2 (grid 2N x 2N), w-stacking over n_wplanes
 *   planes with the same kernel in w.
 *
 * Memory ownership: every pointer argument marked "device" is caller-owned
 * device memory on the job's device (for example a torch tensor's data_ptr());
 * the library never frees it and keeps no reference to it once the call's
 * stream-ordered work has completed.  Everything inside a rix_ctx_t /
 * rix_job_t is library-owned.  Pointers marked "host" are read (or written)
 * before the call returns.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 * are asynchronous unless stated; device errors surface at a later call on
 * the same job or at rix_job_sync.
 *
 * Errors: every call returns RIX_OK (0) or a negative code; rix_last_error()
 * returns a thread-local message for the last failure.  No C++ exception
 * crosses this ABI.
 *
 * Threading: one job must not be used from two host threads at once;
 * different jobs may.
 */
#ifndef RIX_H
#define RIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RIX_MAX_PART 8      /* most uv partitions per job (ring partitions, Sec. 3 generalised) */

#define RIX_OK 0
#define RIX_EINVAL (-1)   /* bad argument, size or pointer */
#define RIX_ENOMEM (-2)   /* device allocation failed or memory budget exceeded */
#define RIX_ECUDA (-3)    /* a CUDA call failed */
#define RIX_ETIMEOUT (-4) /* a bounded device-side wait expired */
#define RIX_ESTATE (-5)   /* calls made out of order (e.g. minor before major) */
#define RIX_EBUSY (-6)    /* the context still owns live jobs */
#define RIX_EINTERNAL (-7) /* a device-side consistency check failed (e.g. a kernel footprint
                              outside the tile its sort key names); results are not trusted */

#define RIX_FP32 0
#define RIX_FP64 1

typedef struct rix_ctx_s* rix_ctx_t;
typedef struct rix_job_s* rix_job_t;
typedef struct rix_batch_s* rix_batch_t;
typedef void* rix_stream_t; /* cudaStream_t */

/* One reconstruction job (Sec. 3: one set of visibilities split into n_part
 * uv partitions, each solved as a pseudo-full-resolution problem). */
typedef struct {
  int32_t n;              /* image side N: power of two, 32 .. 4096 */
  double cell_rad;        /* pixel size (radians), > 0 */
  int32_t n_wplanes;      /* 0 = coplanar; else 9 .. 64 w-planes */
  int32_t nchan;          /* channels per row, 1 .. 65536 */
  const double* freq_hz;  /* host [nchan], copied at rix_job_create */
  int32_t precision;      /* RIX_FP32 or RIX_FP64 */
  int32_t n_part;         /* number of uv partitions: 1 .. RIX_MAX_PART */
  int32_t tile;           /* uv tile side for the sort and the gridder: 16 or 32; 0 = 16 */
  int32_t weighting;      /* RIX_WEIGHT_NATURAL (the given weights) or RIX_WEIGHT_UNIFORM */
  int32_t exchange;       /* RIX_EXCHANGE_IMAGE (0) or RIX_EXCHANGE_SPECTRAL: the form of Phi_p^n */
} rix_job_desc;

/* How a partition's filtered deconvolved residual Phi_p^n = Gamma_p i_bar_p^n
 * travels to the other partitions (Sec. 4.1).  IMAGE: the N x N image.
 * SPECTRAL (the band-limited compression of Sec. 6.3 and Sec. 7 item a):
 * the coefficients of Gamma_p F pad i_bar_p on the ring support of Gamma_p
 * (where Gamma_p > 0) in the half plane k_u <= 0 (i_bar is real, so the
 * spectrum is Hermitian), rix_phi_support of them; the receiver rebuilds the
 * spectrum, its conjugate half, transforms and crops: the same Phi_p up to
 * rounding, in fewer bytes for every partition but the outermost. */
#define RIX_EXCHANGE_IMAGE 0
#define RIX_EXCHANGE_SPECTRAL 1

/* Visibility weighting.  Uniform (Sec. 5.1): each sample's weight is divided
 * by the sum of the weights in its cell of the N x N image's Fourier grid
 * (nearest cell centre, floor(u_lambda N dl + 1/2), likewise v) and in that
 * cell's Hermitian mirror, over the samples inside the grid; the result is
 * held in float32. */
#define RIX_WEIGHT_NATURAL 0
#define RIX_WEIGHT_UNIFORM 1

/* Host-side statistics of a partitioned job (valid after rix_set_uv_partition). */
typedef struct {
  int64_t nrow;
  int64_t n_samples;          /* nrow * nchan */
  int64_t n_outside;          /* samples whose kernel footprint leaves the grid (excluded) */
  int64_t n_entries;          /* sum over partitions of samples in the partition */
  int64_t part_count[RIX_MAX_PART];   /* samples per partition (overlap counted in each) */
  double part_weight[RIX_MAX_PART];   /* weight sum per partition */
  double ell_px[RIX_MAX_PART - 1];    /* ring radii used (pixels of the N-grid's Fourier plane) */
  double delta_px;
  double w_min;               /* lowest w (wavelengths) */
  double dw;                  /* w-plane spacing (wavelengths) */
  double max_dw_nm1;          /* max |dw (n - 1)| over the image (w-stacking accuracy) */
  int32_t window_lo[RIX_MAX_PART];    /* per partition uv-grid window [lo, lo + size) on both axes */
  int32_t window_size[RIX_MAX_PART];
  int64_t n_work_items;       /* gridder work items (tile chunks) over all partitions */
  int32_t cycle[RIX_MAX_PART];        /* major cycles completed per partition */
} rix_job_stats;

/* ms-CLEAN parameters (Eq. 6-7; Sec. 5.2). */
typedef struct {
  const float* scales;        /* host [n_scales], scale radii in pixels, scales[0] = 0 */
  int32_t n_scales;           /* 1 .. 8 */
  double gain;                /* loop gain, (0, 1] */
  int32_t niter;              /* K, maximum CLEAN iterations this cycle */
  double threshold;           /* stop once max |R_0| < threshold */
} rix_msclean_params;

/* FISTA parameters (Eq. 4-5; Sec. 5.2). */
#define RIX_DICT_DB4 0        /* W = the orthonormal periodic Db4 basis */
#define RIX_DICT_DB1_8 1      /* W = [Psi_db1 ... Psi_db8] / sqrt(8), the paper's concatenation of the
                               * first 8 Daubechies wavelets (a tight frame: W W^T = I) */
typedef struct {
  double lambda;              /* > 0: absolute regularisation weight */
  double lambda_rel;          /* used when lambda <= 0: lambda = lambda_rel * max|residual| of cycle 1 */
  int32_t iters;              /* FISTA iterations per major cycle (50 in the paper) */
  int32_t levels;             /* wavelet decomposition levels, 1 .. log2(N) - 3 */
  int32_t dictionary;         /* RIX_DICT_DB4 or RIX_DICT_DB1_8 */
  int32_t reserved;           /* 0 */
  double sched_a, sched_b;    /* sched_a > 0: lambda_n = sched_a * ||residual of cycle n||_2 * sched_b^n
                               * (Sec. 5.2; n = the cycle number from 1), overriding lambda and
                               * lambda_rel; sched_b > 0 */
} rix_fista_params;

/* ---- context and job lifetime --------------------------------------------- */

/* Creates a context on CUDA device `device` that admits jobs while their
 * summed workspace stays within mem_budget_bytes (0 = no budget).  The
 * library's device memory (job buffers and the temporaries of its calls)
 * comes from one stream-ordered pool per device, owned by the library for
 * the life of the process, which keeps up to 8 GiB of freed memory reserved
 * for later calls instead of returning it to the system at every
 * synchronisation. */
int rix_create(rix_ctx_t* ctx, int device, size_t mem_budget_bytes);
/* Destroys a context; RIX_EBUSY while it still owns jobs. */
int rix_destroy(rix_ctx_t ctx);

/* Upper bound of the device memory a job of this shape with `nrow` rows
 * holds (admission control for serving).  Returns 0 for an invalid desc. */
size_t rix_job_workspace_bytes(const rix_job_desc* desc, int64_t nrow);

/* Validates desc and creates an empty job; RIX_ENOMEM if the context budget
 * cannot admit rix_job_workspace_bytes(desc, max_rows). */
int rix_job_create(rix_ctx_t ctx, const rix_job_desc* desc, int64_t max_rows, rix_job_t* job);
/* Waits for the work the job's calls issued (on every stream they used, not
 * for other jobs), then releases the job's device memory without
 * synchronising the device. */
int rix_job_destroy(rix_job_t job);
/* Blocks until the work issued by the job's calls has finished (other jobs'
 * work is not waited for) and reports deferred device errors. */
int rix_job_sync(rix_job_t job);
int rix_job_get_stats(rix_job_t job, rix_job_stats* out);

/* ---- a1-a3: coordinates, partition, tile sort (Sec. 3, Fig. 3) ------------- */

/* Computes each sample's grid coordinates (FP64), its radius
 * r = |(u, v)|_lambda N dl in pixels of the N-grid's Fourier plane, and its
 * partitions: sample in p  <=>  (p == 0 or r >= ell_p - delta) and
 * (p == n_part-1 or r <= ell_{p+1} + delta), both inclusive (overlapping
 * domains of Sec. 3).  ell_px: host [n_part-1] ascending ring radii, or NULL
 * for the lower i/n_part quantiles of r over all samples (element
 * floor(i (n-1) / n_part) of the ascending order; the lower median for 2).
 * delta_px: overlap half-width (1 pixel in Sec. 5.1).  Samples whose kernel
 * footprint leaves the grid are excluded and counted.  Then sorts the
 * (sample, partition) entries stably by the key (partition, first w-plane,
 * tile row, tile column) with an LSD radix sort and builds the gridder's
 * work items.
 *   uvw_m    device [nrow][3] float64, copied into the job
 *   weight   device [nrow][nchan] float32 or NULL (= 1), copied
 *   mask_out device [nrow][nchan] uint8 or NULL: bit p set for partition p
 *            (0 for excluded samples)
 * Synchronises `stream` once at the end (sizes are read back to the host).
 * May be called again to re-partition; resets every partition's state. */
int rix_set_uv_partition(rix_job_t job, const double* uvw_m, int64_t nrow, const float* weight,
                         const double* ell_px, double delta_px, uint8_t* mask_out,
                         rix_stream_t stream);

/* Copies the weights the job images with ([nrow][nchan] float32, after the
 * job's weighting; 1 for natural weighting without given weights) to the
 * device buffer weight_out.  Needs rix_set_uv_partition. */
int rix_get_weights(rix_job_t job, float* weight_out, rix_stream_t stream);

/* Copies the sorted entries (keys and sample indices, rix_job_stats.n_entries
 * of each) to device buffers; keys are packed as
 * part << (2 bt + bw) | plane << 2 bt | tile_row << bt | tile_col with
 * bt = log2(2N / tile) and bw = bits of (n_wplanes - 7) (0 if coplanar). */
int rix_get_sorted_entries(rix_job_t job, uint32_t* keys_out, uint32_t* samples_out,
                           rix_stream_t stream);

/* ---- a4-a7: the measurement operator (Eq. 2) ------------------------------- */

/* Degridding G^dagger F (Eq. 2): model visibilities of `image` (device N x N)
 * for the samples of partition `part`, written to vis_out (device
 * [nrow][nchan] complex); samples outside the partition are left untouched. */
int rix_degrid(rix_job_t job, int part, const void* image, void* vis_out, rix_stream_t stream);

/* Gridding F^dagger G (Eq. 2): dirty image Re(A^H (w . vis)) / W_part of the
 * partition's samples (device vis [nrow][nchan] complex) into image_out
 * (device N x N). */
int rix_grid(rix_job_t job, int part, const void* vis, void* image_out, rix_stream_t stream);

/* PSF of partition `part`: the dirty image of unit visibilities on a 2N x 2N
 * image (centre at pixel (N, N)), normalised by the weight sum W_part, into
 * psf_out (device (2N)^2, may be NULL); *weight_sum_out (host, may be NULL)
 * receives W_part.  Computed once and kept by the job. */
int rix_psf(rix_job_t job, int part, void* psf_out, double* weight_sum_out, rix_stream_t stream);

/* How rix_psf forms the 2N x 2N PSF (both approximate Re A^H w / W_part of
 * Sec. 2's measurement operator to the gridding kernel's accuracy):
 *   RIX_PSF_DOUBLE_GRID  one gridding of the unit visibilities on the 2N
 *                        image's own oversampled grid (side 2 Ng = 4N);
 *   RIX_PSF_TILES        four N x N tiles on the image grid (side Ng): tile t
 *                        is the dirty image of exp(2 pi i (u l_t + v m_t))
 *                        with its image-domain factors taken at the sky
 *                        positions of its pixels (shift theorem); the PSF
 *                        grid is never formed, so it serves N = 4096 (FP32)
 *                        and N = 2048 (FP64), whose 4N-long transforms exceed
 *                        the transform passes' limit;
 *   RIX_PSF_AUTO         (default) DOUBLE_GRID when 4N is within that limit,
 *                        else TILES.
 * Setting a method drops the job's PSFs (they are formed again, lazily).
 * Host-only; RIX_EINVAL for an unknown method. */
#define RIX_PSF_AUTO 0
#define RIX_PSF_DOUBLE_GRID 1
#define RIX_PSF_TILES 2
int rix_job_set_psf_method(rix_job_t job, int32_t method);

/* One major cycle of partition `part` (Eq. 2): residual
 * F^dagger G (v - G^dagger F model) / W_part of the partition's samples, with
 * degrid, residual and grid fused per tile.  vis_obs: device [nrow][nchan]
 * complex observed visibilities.  model: device N x N to replace the job's
 * resident model image of the partition first, or NULL to use the resident
 * model (zero initially; the minor cycles add to it, Eq. 3).  residual_out:
 * device N x N or NULL.  Advances the partition's cycle counter. */
int rix_major_cycle(rix_job_t job, int part, const void* vis_obs, const void* model,
                    void* residual_out, rix_stream_t stream);

/* ---- a8-a10: fill and minor cycles (Sec. 4, Eq. 4-7) ---------------------- */

/* Minor cycle of partition `part` at its current cycle n, by multi-scale
 * CLEAN on the pseudo-full-resolution problem of Eq. 7: first adds the other
 * partitions' filtered deconvolved residuals Phi_q^{n-1} to the aggregates
 * rho_{q->p} (n >= 2), builds the dirty image
 *   gamma Gamma_p i_p + sum_q mu_q H_q rho_{q->p}
 * and PSF gamma Gamma_p H_p + sum_q mu_q Gamma_q H_q ((gamma, mu) = (1, 0) at
 * n = 1, else the partitions' weight fractions), cleans it (scales limited to
 * those present in the partition at n = 1), then updates the resident model
 * (Eq. 3), publishes Phi_p^n = Gamma_p i_bar_p^n and subtracts
 * Gamma_q i_bar_p^n from rho_{q->p}.  delta_out: device N x N or NULL,
 * receives i_bar_p^n.  Needs the major cycle n of `part` and the minor cycle
 * n-1 of every partition (RIX_ESTATE otherwise). */
int rix_minor_cycle_msclean(rix_job_t job, int part, const rix_msclean_params* params,
                            void* delta_out, rix_stream_t stream);

/* Same for the sparsity-regularised minor cycle of Eq. 5 (Eq. 4 when
 * n_part = 1): FISTA on
 *   ||Gamma_p (i_p - H_p W alpha)||^2 + gamma_n sum_q ||rho_{q->p} - Gamma_q W alpha||^2
 *   + lambda ||alpha||_1
 * with W the orthonormal periodic Db4 wavelet basis or the concatenation of
 * db1 .. db8 (params->dictionary), gamma_n = 0 at n = 1 and 1 afterwards. */
int rix_minor_cycle_fista(rix_job_t job, int part, const rix_fista_params* params,
                          void* delta_out, rix_stream_t stream);

/* The FISTA minor cycles of several partitions of the same cycle, with the
 * same parameters, as one launch of the iteration loop: equivalent to
 * rix_minor_cycle_fista for parts[0], ..., parts[n_parts - 1] in turn
 * (without delta_out), with the same call-order rules for each.  parts: host
 * array of n_parts distinct partition indices, 1 <= n_parts <= n_part.  Each
 * partition's preparation (fill tables) and finish (image update, exchange
 * terms) run on a stream the job owns, after the caller's work on `stream`
 * and after that partition's own major cycle and the other partitions'
 * previous minor cycles, whatever streams those ran on; the loop runs on
 * `stream`, which on return waits for all of it.  With the Db4 dictionary
 * the loops of the batch run as a dataflow (each phase of a loop waits only
 * for the previous phase of the same loop, so one loop's phase ends are
 * filled with the others' work); with the concatenated dictionary they
 * advance together, one grid barrier per phase serving all of them.  Every
 * device-side wait is bounded (RIX_ETIMEOUT at rix_job_sync). */
int rix_minor_cycle_fista_batch(rix_job_t job, int n_parts, const int32_t* parts, const rix_fista_params* params,
                                rix_stream_t stream);

/* ms-CLEAN components found by the last minor cycle of `part`: count (host)
 * and, when non-NULL, up to `capacity` entries of scale index and row-major
 * pixel index (host int32) and amplitude (host double), in the order found.
 * Synchronises the stream. */
int rix_get_components(rix_job_t job, int part, int32_t* count, int32_t capacity,
                       int32_t* scale_out, int32_t* pixel_out, double* amp_out,
                       rix_stream_t stream);

/* Copies the resident model image of `part` (device N x N). */
int rix_get_model(rix_job_t job, int part, void* image_out, rix_stream_t stream);

/* ---- a11: combine (Sec. 5.2) ----------------------------------------------- */

/* Final image: the equal-weight mean of the partitions' model images
 * (0.5 / 0.5 for two partitions), device N x N. */
int rix_combine(rix_job_t job, void* image_out, rix_stream_t stream);

/* ---- batched major cycles and gridder tuning ------------------------------ */

/* Tuning of the FP32 w-stacked gridder of a job (a deployment knob; the paper
 * has no counterpart): chunk_limit (1 .. 256) = the most samples with one
 * kernel footprint a warp grids between two flushes of its accumulators
 * (the work items' entries are regrouped on the spot when it changes;
 * results are the same up to rounding), ctas_per_sm (0 .. 8, 0 = as many as
 * fit) = resident gridder CTAs per SM.  Defaults 64 and 0.  Waits for the
 * job's own work. */
int rix_job_tune(rix_job_t job, int32_t chunk_limit, int32_t ctas_per_sm);

/* A batch of (job, partition) pairs whose major cycles run together (the
 * paper's independent partition jobs, Sec. 3, for many jobs at once): every
 * pair's model -> w-planes transform, then ONE persistent gridder launch over
 * all pairs' work items (degrid, residual, grid of Eq. 2), then every pair's
 * planes -> residual transform.  jobs: host [n] (FP32 w-stacked, tile 16,
 * partitioned, of this context); parts: host [n]; pairs distinct.  The batch
 * records the pairs' buffers: create it after rix_set_uv_partition and
 * rix_job_tune, and again after re-partitioning a job; the jobs outlive it.
 * Allocates the pairs' plane buffers if needed and uploads the gridder's
 * per-pair descriptors (synchronises the device). */
int rix_batch_create(rix_ctx_t ctx, int32_t n, const rix_job_t* jobs, const int32_t* parts, rix_batch_t* batch);
int rix_batch_destroy(rix_batch_t batch);

/* One major cycle of every pair, as rix_major_cycle(jobs[i], parts[i],
 * vis_obs[i], NULL, NULL) for each (the same call-order rules and result:
 * the residual stays resident for the partition's minor cycle, the cycle
 * counters advance).  vis_obs: host [n] of device pointers [nrow][nchan]
 * float2.  residual_out: NULL, or host [n] of device pointers (N x N float,
 * NULL entries skipped) that receive the pairs' residual images.  The
 * pairs' transforms run on streams of the batch forked from
 * and joined to `stream`; nothing is allocated or synchronised, so the
 * call can be captured in a CUDA graph once the pairs have run one
 * (uncaptured) major cycle.  A captured call is not an executed one: it
 * waits on and records none of the jobs' events and leaves their cycle
 * counters as they were, so a replayed graph repeats the captured cycle
 * (on the models of the moment) and its ordering against other work is the
 * caller's. */
int rix_batch_major_cycle(rix_batch_t batch, const void* const* vis_obs, void* const* residual_out,
                          rix_stream_t stream);

/* Device time of the FP32 w-stacked gridder on one partition (a tuning
 * diagnostic): the mean over `reps` launches of the residual mode (degrid,
 * residual, grid) with the job's current tuning, on the partition's plane
 * buffers, which hold nothing between major cycles; the job's results and
 * cycle state are untouched.  vis_obs: device [nrow][nchan] float2.  Waits
 * for the job's work and synchronises. */
int rix_gridder_probe(rix_job_t job, int part, const void* vis_obs, int32_t reps, double* ms_out);

/* Device time of partition `part`'s fused major-cycle operator (a
 * measurement diagnostic): model -> w-planes, degrid, residual and grid,
 * planes -> residual image (Eq. 2), on the partition's current resident
 * model, into a temporary image; the mean over `reps` runs after one
 * untimed run.  The job's results and cycle state are untouched (no call
 * order is needed); allocates one image; waits for the job's work and
 * synchronises. */
int rix_major_cycle_probe(rix_job_t job, int part, const void* vis_obs, int32_t reps, double* ms_out);

/* ---- band-limited exchange (Sec. 6.3, Sec. 7 item a) ---------------------- */

/* Number of complex coefficients of partition `part`'s band-limited
 * message (valid after rix_set_uv_partition; fixed for the job): the points
 * of the centred 2N x 2N frequency grid with Gamma_part > 0 and k_u <= 0. */
int rix_phi_support(rix_job_t job, int part, int64_t* count_out);

/* The band-limited message of partition `part`'s last minor cycle: the
 * coefficients of Gamma_part F pad i_bar (i_bar the deconvolved residual of
 * that cycle) at the rix_phi_support points, in ascending order of the
 * u-major flat index ju * 2N + jv (ju, jv the centred indices of k_u, k_v),
 * into packed_out (device, the job precision's complex type).  Needs a
 * completed minor cycle of the partition (RIX_ESTATE otherwise). */
int rix_phi_pack(rix_job_t job, int part, void* packed_out, rix_stream_t stream);

/* Phi = crop F^-1 of the spectrum rebuilt from such coefficients of
 * partition `part` (their conjugates completing the other half plane),
 * normalised like the minor cycles' filtered images: into phi_out (device
 * N x N real).  The round trip rix_phi_pack -> rix_phi_unpack gives
 * Gamma_part i_bar without loss beyond rounding. */
int rix_phi_unpack(rix_job_t job, int part, const void* packed, void* phi_out, rix_stream_t stream);

/* ---- baseline-dependent averaging (Sec. 6.2, Sec. 7 item d) ---------------- */

/* The remedy the paper names for unbalanced partitions: a dense uv centre
 * (Sgr B2, Sec. 6.2) leaves the outer partition idle; averaging each
 * baseline's consecutive time samples over a window that shrinks with its
 * uv speed (after Wijnholds et al. 2018) thins the centre, so a ring radius
 * splits the samples more evenly.  A preprocessing step before
 * rix_set_uv_partition, on the context's device.
 *   uvw_m    device [n_times][n_baselines][3] float64, rows time-major
 *   vis      device [n_times * n_baselines][nchan] complex (float2 for
 *            RIX_FP32, double2 for RIX_FP64)
 *   weight   device [n_times * n_baselines][nchan] float32, or NULL (= 1)
 *   freq_hz  host [nchan]
 * Per baseline b: s_b = the largest (u, v) change between consecutive times
 * at the highest frequency, in cells of the N x N image's Fourier grid
 * (|du, dv|_lambda N cell_rad, the unit of the partition radius); window
 * k_b = min(n_times, max(1, floor(max_shift_px / s_b))) time samples
 * (n_times when s_b = 0); the times are cut into consecutive windows of k_b,
 * the last shorter.  Each window gives one output row: the mean uvw, and per
 * channel the weight sum and the weighted mean visibility (0 when the sum
 * is 0).  Output rows are baseline-major (baseline 0's windows in time
 * order, then baseline 1's, ...).  The window arithmetic is FP64 with every
 * product, sum and quotient rounded separately; sums are FP64. */

/* The number of averaged rows (host *nrow_out) and optionally the windows
 * k_b (host [n_baselines] int32).  Synchronises `stream`. */
int rix_bda_rows(rix_ctx_t ctx, const double* uvw_m, int64_t n_times, int64_t n_baselines, const double* freq_hz,
                 int32_t nchan, int32_t n, double cell_rad, double max_shift_px, int32_t* window_out,
                 int64_t* nrow_out, rix_stream_t stream);

/* The averaged rows into uvw_out (device [rows][3] float64), vis_out (device
 * [rows][nchan], the precision's complex type) and weight_out (device
 * [rows][nchan] float32); RIX_EINVAL when they hold fewer than the rows
 * rix_bda_rows reports (nrow_capacity).  *nrow_out (host, may be NULL)
 * receives the row count.  Synchronises `stream` once (the row count is read
 * back) before the averaging kernel is queued. */
int rix_bda_average(rix_ctx_t ctx, const double* uvw_m, const void* vis, const float* weight, int64_t n_times,
                    int64_t n_baselines, const double* freq_hz, int32_t nchan, int32_t precision, int32_t n,
                    double cell_rad, double max_shift_px, double* uvw_out, void* vis_out, float* weight_out,
                    int64_t nrow_capacity, int64_t* nrow_out, rix_stream_t stream);

/* ---- gridding without device allocation ----------------------------------- */

/* rix_grid for callers that cannot allocate device memory while they grid:
 * a host loop with a latency budget that must not stall on the allocator
 * (cudaMalloc and cudaFree can synchronise the device), a process whose
 * device memory another allocator has already reserved, or a host program
 * that does not let a library own device allocations.  The paper has no
 * counterpart; this is a deployment variant of rix_grid.
 *
 * Same arguments, layout and result as rix_grid (FP32 jobs only).  The
 * partition's w-planes and transpose buffer live in one scratch area of
 * RIX_GRID_NOALLOC_MAX_BYTES compiled into the library as a device array:
 * every GPU that loads the library holds it until the process exits.  A
 * partition needing more (max(n_wplanes, 1) * S * (S + N) * 8 bytes, S = its
 * uv window side from rix_job_get_stats) is rejected with RIX_EINVAL; the
 * scratch left over holds the plane-group images of the inverse transform
 * (fewer groups, down to one, when little is left: the result is the same).
 * The call allocates no device memory (rix_device_allocations does not move
 * across it); it zeroes the part of the scratch it accumulates into, so each
 * call starts clean, but all calls share the one scratch: calls whose GPU
 * work overlaps in time (other streams, other threads, other jobs) race and
 * corrupt each other's results.  The first call on a device looks up the
 * scratch's device address (once per device, with that device current) and
 * keeps it for the life of the process, which assumes the device's primary
 * context is never reset (no cudaDeviceReset before a later call); make that
 * first call before any stream capture.  The call runs on the job's device
 * and leaves the caller's current device as it found it.  It records
 * `stream` with the job, so rix_job_destroy waits for its work.  The job
 * itself (rix_job_create, rix_set_uv_partition) is set up beforehand as
 * usual. */
#define RIX_GRID_NOALLOC_MAX_BYTES (32u << 20)
int rix_grid_noalloc(rix_job_t job, int part, const void* vis, void* image_out, rix_stream_t stream);

/* Number of device allocations the library has made in this process (every
 * one is a stream-ordered pool allocation; a diagnostic: the difference
 * across a call sequence is that sequence's allocation count). */
uint64_t rix_device_allocations(void);

/* Thread-local message of the last failed call on this thread. */
const char* rix_last_error(void);

/* Number of CUDA kernels the library has run in this process, over all jobs
 * and host threads, counting each kernel node of a replayed CUDA graph (a
 * diagnostic: the difference across a call sequence is that sequence's
 * kernel count). */
uint64_t rix_kernel_launches(void);

/* Opt-in device timing (a diagnostic for benchmarks): while enabled, the
 * library records CUDA events on the launch stream around every launch of
 * the kernel classes below (launches inside stream captures are not timed).
 * rix_timing_read waits for the recorded events and returns, for one class,
 * the summed launch durations (ms), the busy time (ms: the union of the
 * launch intervals, which differs from the sum when launches on different
 * streams overlap) and the number of launches, then clears them.
 * Classes: 0 = tiled degrid/grid kernel, 1 = FFT passes, 2 = partition,
 * 3 = minor-cycle loop kernels. */
#define RIX_TIME_TILES 0
#define RIX_TIME_FFT 1
#define RIX_TIME_PARTITION 2
#define RIX_TIME_MINOR_LOOP 3   /* the persistent FISTA loop and the ms-CLEAN kernel */
int rix_timing_enable(int on);
int rix_timing_read(int kernel_class, double* total_ms, double* busy_ms, int64_t* launches);

/* The Daubechies low-pass filter with p vanishing moments (p in 1 .. 8) that
 * the concatenated dictionary uses: writes its 2p taps to h_out (host memory,
 * room for 2p doubles), minimum phase, sum sqrt(2), and returns 2p (a
 * negative RIX_E* code on bad arguments).  Host-only; no device needed. */
int rix_daubechies_lowpass(int p, double* h_out);

/* Self-test of the failure-detection path (a diagnostic; the paper has no
 * counterpart).  Launches, on the context's device, a cooperative kernel of
 * one CTA per SM whose first CTA never arrives at the library's bounded grid
 * barrier: every other CTA's wait runs out (after about 2 s), the first one
 * to give up stores RIX_ETIMEOUT in a status word, all of them return, and
 * the call synchronises.  *status_out receives the status word (RIX_ETIMEOUT
 * when detection works) and *gave_up_out the number of CTAs that left the
 * barrier without it completing (all but one).  Returns RIX_OK when the
 * kernel ran to completion, whatever the status; the context stays usable.
 * Blocks the calling thread for the length of the wait. */
int rix_selftest_barrier_timeout(rix_ctx_t ctx, int* status_out, int* gave_up_out);

#ifdef __cplusplus
}
#endif
#endif /* RIX_H */
