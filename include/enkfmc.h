/*
 * enkfmc.h -- C ABI of the GB300 EnKF-MC analysis library (libenkfmc.so).
 *
 * EnKF-MC is the stochastic ensemble Kalman filter whose inverse background
 * covariance is estimated by a localised modified Cholesky decomposition
 * (Nino, Sandu, Deng 2016).  One analysis step runs in three calls:
 *
 *   enkfmc_estimate   regress every component on its predecessors inside the
 *                     local box of radius r (Section 2.1 Eq. 1-3, Section 2.3
 *                     Eq. 8): one row of the unit lower triangular T and one
 *                     entry of the diagonal D per component.
 *   enkfmc_assemble   per sub-domain extended by an r-wide boundary (Section 3,
 *                     Algorithm 3): re-estimate the boundary rows from the local
 *                     samples, assemble A = T^T D^-1 T + H^T R^-1 H (Eq. 11) and
 *                     factor A = L L^T.
 *   enkfmc_analyze    form the perturbed observations, solve A dX = H^T R^-1
 *                     (Y^s - H X^b) for all N members (Eq. 11) and write the
 *                     interior of every sub-domain into X^a = X^b + dX (Eq. 10,
 *                     Algorithm 2).
 *
 * Conventions shared by every call
 *   - Floating-point arrays hold `double` when the handle's precision is
 *     ENKFMC_FP64 and `float` otherwise.  Index arrays are int32/int64 as
 *     declared.
 *   - Ensembles are member-major: X[m * n + l] is member m (0 <= m < N) of the
 *     component with label l.  Labels are variable-major: 3-D variables first
 *     (nlev levels each), then 2-D variables (one level); within a variable
 *     l = offset(v) + (level * nlat + lat) * nlon + lon.
 *   - Unless a parameter says "host", pointers are device pointers owned by
 *     the caller; the library never frees them and keeps no reference after
 *     the call returns, except that enkfmc_assemble reads Tvals and D again in
 *     later enkfmc_analyze calls (they must stay valid and unchanged until the
 *     next enkfmc_assemble).
 *   - The handle owns its tables, factors and workspace (device memory
 *     allocated by enkfmc_create / enkfmc_set_observations, released by
 *     enkfmc_destroy).
 *   - Calls are asynchronous on the handle's CUDA stream.  Argument errors are
 *     returned synchronously.  Numerical failures (a Gram matrix or a
 *     sub-domain matrix that is not positive definite, a residual variance
 *     <= 0, a non-finite value) are recorded on the device and reported by
 *     enkfmc_get_status, which synchronises the stream.  No kernel traps.
 *   - A handle is not re-entrant: calls on one handle must not overlap.
 */
#ifndef ENKFMC_H
#define ENKFMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ENKFMC_OK = 0,
  ENKFMC_EINVAL = 1,     /* invalid argument or unsupported geometry            */
  ENKFMC_ENOMEM = 2,     /* device or host allocation failed                     */
  ENKFMC_ENOTSPD = 3,    /* a sub-domain matrix A is not positive definite       */
  ENKFMC_EDNONPOS = 4,   /* a Gram matrix is singular or a variance D_j <= 0     */
  ENKFMC_ENONFINITE = 5, /* NaN or Inf met                                        */
  ENKFMC_ETIMEOUT = 6,   /* a bounded device wait ran out                         */
  ENKFMC_ECUDA = 7,      /* a CUDA runtime call failed                            */
  ENKFMC_ENOTIMPL = 8,   /* not implemented                                       */
  ENKFMC_ESTATE = 9      /* call out of order (e.g. analyze before assemble)      */
} enkfmc_status;

typedef enum {
  ENKFMC_FP64 = 0,       /* every step in double precision                        */
  ENKFMC_FP32 = 1        /* single precision arithmetic with iterative refinement:
                            one step per regression (corrected semi-normal
                            equations, residual of the anomalies), and per
                            sub-domain solve (Eq. 11) one or more steps whose
                            residuals are accumulated in compensated
                            (double-float) arithmetic.  Rows with more
                            predecessors than half the members (2p > N, nearly
                            singular Gram matrices) are regressed in double
                            precision from FP64 anomalies and FP64 covariances
                            of the single-precision ensemble; their T and D are
                            stored in single precision like every other row    */
} enkfmc_precision;

/* enkfmc_problem.flags */
enum {
  ENKFMC_FLAG_NO_SOLVE_REFINEMENT = 1, /* FP32: skip the sub-domain refinement step
                                          (the plain single-precision solve)      */
  ENKFMC_FLAG_REFINE_MASK = 0xF00,     /* FP32: bits 8-11 (ENKFMC_FLAG_REFINE_STEPS(k))
                                          = refinement steps of every sub-domain
                                          solve, 1-15; 0 = one step, or four when
                                          some row has 2p > N (ill-conditioned A);
                                          the reverse pass refines its solve alike */
  ENKFMC_FLAG_PLAIN_FP32 = 4,          /* FP32: the plain single-precision form of the
                                          statistics and factorisations: every row
                                          regressed in single precision (also where
                                          2p > N) and no double-precision blocks (a
                                          block whose single-precision factorisation
                                          meets a non-positive pivot reports
                                          ENKFMC_ENOTSPD); with
                                          ENKFMC_FLAG_NO_SOLVE_REFINEMENT the whole
                                          path is plain FP32.  For comparison with
                                          the mixed-precision default              */
  ENKFMC_FLAG_SIMT_BAND = 2            /* FP32: take the band Cholesky and the band
                                          solves on the CUDA cores only.  By
                                          default their rank-32 panel updates run
                                          on the tensor cores as three TF32
                                          products of a hi + lo split of each
                                          operand (about 21 significant bits per
                                          product, FP32 accumulation), when the
                                          band fits (half-width < 384; for the
                                          solves also N <= 128); FP64 always uses
                                          the CUDA cores                           */
};

#define ENKFMC_FLAG_REFINE_STEPS(k) ((int32_t)(k) << 8)

/* Problem description.  Neighbours of a component share its variable, lie
 * within `vert_reach` levels and within Chebyshev distance r on the
 * (lat, lon) grid, longitude taken on the ring when lon_periodic != 0
 * (Section 2.2, local boxes of Fig. 1).  Predecessors are the neighbours with
 * a smaller label (Section 2.3, Fig. 2).  Sub-domains are sub_lat x sub_lon
 * column tiles from (0, 0), the last ones ragged, extended by r columns on
 * every side (clipped at the poles, wrapped in longitude) (Section 3).
 * Requirements: nlon >= 2r+1 when lon_periodic, 2 <= N <= 128,
 * nvar_3d + nvar_2d <= 16, r <= 16, fewer than 2^31 components, at most 255
 * stencil slots per row (pmax).
 * An extended sub-domain as wide as the ring covers it exactly once.  */
typedef struct {
  int32_t nlon, nlat, nlev, nvar_3d, nvar_2d;
  int32_t lon_periodic;
  int32_t r;
  int32_t vert_reach;
  int32_t N;
  int32_t sub_lon, sub_lat;
  int32_t precision;     /* enkfmc_precision                                      */
  double ridge_c;        /* lambda = ridge_c * tr(G) / p wherever p >= N - 1      */
  int32_t flags;         /* ENKFMC_FLAG_* bits, 0 by default                      */
} enkfmc_problem;

/* Sizes of a created handle (host struct filled by enkfmc_query). */
typedef struct {
  int64_t n;             /* number of components                                  */
  int32_t pmax;          /* slots per T row in the stencil layout of Tvals        */
  int32_t nsub;          /* sub-domains                                           */
  int32_t nblock;        /* (sub-domain, variable) blocks of A                    */
  int32_t hb_max;        /* largest half-bandwidth of a block of A                */
  int64_t ext_rows;      /* components in all extended sub-domains                */
  int64_t halo_rows;     /* boundary rows re-estimated by enkfmc_assemble         */
  int64_t band_elems;    /* stored band entries of all blocks of A                */
  int64_t workspace_bytes;
  int64_t m;             /* observations set by enkfmc_set_observations (or -1)   */
  int32_t tc_chol;       /* 1: band Cholesky updates on the tensor cores          */
  int32_t tc_solve;      /* 1: band solve panel updates on the tensor cores       */
  int32_t refine_steps;  /* refinement steps of every sub-domain solve            */
  int32_t fp64_rows;     /* 1: rows with 2p > N regressed in double precision     */
} enkfmc_info;

typedef struct enkfmc_handle enkfmc_handle;

/* Create a handle for one problem on the current CUDA device.  `cuda_stream`
 * is a cudaStream_t (NULL = legacy default stream).  Builds the geometry
 * tables and allocates the workspace.  Returns EINVAL for unsupported
 * geometry, ENOMEM when device memory runs out.  Unsupported includes a band
 * of A (half-width about the tile's extended area per level times the levels
 * a row reaches) wider than the CUDA-core band kernels hold in shared memory:
 * about 620 in double precision, which FP64 problems and the double-precision
 * blocks of FP32 problems use, and 1,280 in single precision. */
enkfmc_status enkfmc_create(enkfmc_handle** h, const enkfmc_problem* p, void* cuda_stream);
void enkfmc_destroy(enkfmc_handle* h);
/* Validate a problem description without a device: OK, or EINVAL where
 * enkfmc_create would refuse it as invalid or unsupported (except the band
 * width, which enkfmc_create checks once it has built the sub-domains). */
enkfmc_status enkfmc_check_problem(const enkfmc_problem* p);
const char* enkfmc_strerror(enkfmc_status s);
enkfmc_status enkfmc_query(const enkfmc_handle* h, enkfmc_info* info /* host */);
enkfmc_status enkfmc_set_stream(enkfmc_handle* h, void* cuda_stream);

/* Stencil layout of Tvals: slot s of a row holds the coefficient of the
 * neighbour at offset (dk[s], dlat[s], dlon[s]) (longitude offset taken on
 * the ring), or 0 when that neighbour is not a predecessor.  Host arrays of
 * length pmax. */
enkfmc_status enkfmc_slot_offsets(const enkfmc_handle* h, int32_t* dk, int32_t* dlat,
                                  int32_t* dlon);

/* Observation network H: obs_idx (host, length m) lists the observed
 * component labels in increasing order, without repeats (H selects
 * components, Section 2.3).  Synchronous; validates and uploads index
 * tables.  Must precede enkfmc_assemble.  m = 0 is allowed (no update). */
enkfmc_status enkfmc_set_observations(enkfmc_handle* h, const int32_t* obs_idx, int64_t m);

/* Step (a), Eq. 1-3 and Eq. 8 with S = U^b (Eq. 5): anomalies of Xb
 * ([N][n]), then for every component j the regression on its predecessors:
 * Tvals[j * pmax + s] = -beta (0 for absent slots) and D[j] = residual sum of
 * squares / (N - 1).  Tvals: [n][pmax], D: [n], written on the stream. */
enkfmc_status enkfmc_estimate(enkfmc_handle* h, const void* Xb, void* Tvals, void* D);

/* Step (b), Algorithm 3 and Eq. 11: for every sub-domain re-estimate the
 * boundary rows of its extended set from the local samples (predecessors
 * cut to the extended set), assemble A = T^T D^-1 T + H^T R^-1 H in band
 * storage per (sub-domain, variable) block and factor it.  In single
 * precision a block whose factorisation meets a non-positive pivot (a
 * condition number beyond what single precision holds) is assembled again
 * from the same T and D in double precision and factored, and later solved,
 * in double; ENOTSPD is reported only if that fails too.  (The handle holds
 * room for every block in double precision: twice the band's bytes.)  Xb: [N][n]
 * (when it is the same pointer as in the last enkfmc_estimate on this
 * handle, the anomalies and covariances computed there are reused, so its
 * contents must not change in between);
 * Tvals, D: as written by enkfmc_estimate; Rdiag: [m] observation-error
 * variances.  Requires enkfmc_set_observations. */
enkfmc_status enkfmc_assemble(enkfmc_handle* h, const void* Xb, const void* Tvals,
                              const void* D, const void* Rdiag);

/* Step (c), Eq. 10-11 and Algorithm 2: Y^s = y 1^T + diag(sqrt(R)) Z^T with
 * Z [N][m] standard normals; dX = A^-1 H^T R^-1 (Y^s - H X^b) per sub-domain
 * (in single precision refined, and with three or more refinement steps a
 * block whose corrections predict an error above 1e-6 of its solution after
 * the second step is factored and solved in double precision from there);
 * Xa[m * n + l] = Xb + dX for l in the sub-domain's interior.  Xb, Xa:
 * [N][n] (Xa may not alias Xb); y, Rdiag: [m]; Z: [N][m].  Uses the factors
 * of the last enkfmc_assemble. */
enkfmc_status enkfmc_analyze(enkfmc_handle* h, const void* Xb, const void* y,
                             const void* Rdiag, const void* Z, void* Xa);

/* Steps (b) and (c) in the dual form, Eq. 12-13: per (sub-domain, variable)
 * block, with the block's T (boundary rows re-estimated from the local
 * samples, as in enkfmc_assemble) and D, and the m_b observations inside its
 * extended set,
 *   Z = T^-T H^T (n_b x m_b),   (R + Z^T D Z) W = Y^s - H X^b (m_b x N),
 *   dX = T^-1 D Z W  =  X~ V^T (R + V V^T)^-1 (Y^s - H X^b),
 * with T X~ = D^1/2 and V = H X~; Xa = Xb + dX on the interiors.  The same
 * analysis as enkfmc_assemble + enkfmc_analyze (exactly, up to rounding),
 * without the band matrix: its cost grows with m_b instead of the band, so it
 * is the cheaper form for sparse networks.  Arguments as for enkfmc_assemble
 * and enkfmc_analyze (Tvals, D from enkfmc_estimate; Xb the same ensemble).
 * Arithmetic: the problem's precision, except single-precision problems with
 * rows where 2p > N (the regressions' double-precision rule), whose dual
 * arithmetic is double (their T^-1 and R + Z^T D Z lose the single-precision
 * digits; inputs and Xa stay single precision).  Requires
 * enkfmc_set_observations.  Returns EINVAL, with nothing queued, when a
 * block's observation system (m_b (m_b + 1) / 2 + max(m_b N, 32 m_b)
 * elements; m_b up to about 260 at N = 80 in single precision) or a
 * triangular solve's ring ((vr ey + r + 1) ex rows of 32 elements, ey x ex
 * the extended box) exceeds 227 KB of shared memory, or the stencil has more
 * than 128 slots; ENOTSPD (status) when
 * R + Z^T D Z is not positive definite for a block in the arithmetic (its
 * increment is then zero): with rows where p nears N - 1 and no ridge, T^-1
 * can grow beyond even double precision's range (entries of 1e12 at
 * N = 40, p = 37), where the primal form applies.  A refusal (EINVAL)
 * changes nothing on the handle; after a dual analysis enkfmc_analyze needs a
 * new enkfmc_assemble, and enkfmc_analyze_adjoint does not apply to it. */
enkfmc_status enkfmc_analyze_dual(enkfmc_handle* h, const void* Xb, const void* Tvals,
                                  const void* D, const void* y, const void* Rdiag,
                                  const void* Z, void* Xa);

/* One full analysis from HOST buffers (same layouts as above): copies the
 * inputs to the device, runs estimate + assemble + analyze, copies Xa back,
 * and synchronises.  Returns the first numerical status as well.  y, Rdiag
 * and Z are copied on a second stream of the handle while the estimate runs
 * (page-locked host buffers let the copies overlap it); no copy is in flight
 * when the call returns, on success or error. */
enkfmc_status enkfmc_cycle_host(enkfmc_handle* h, const void* Xb, const void* y,
                                const void* Rdiag, const void* Z, void* Xa);

/* ---------------------------------------------------------------------------
 * Filter cycling (Algorithm 1: analysis, then the model step of every member,
 * repeated while observations arrive).  The paper's model (SPEEDY) is
 * replaced by a synthetic forecast operator, and the analysis error is the
 * RMSE of Eq. 18.
 * ------------------------------------------------------------------------ */
/* Forecast operator: every field of nvec state vectors (device, member-major
 * [nvec][n], the handle's element type) moves `shift` cells eastward along its
 * latitude circle, periodic in longitude (advection of the random fields,
 * whose statistics it keeps), with multiplicative covariance inflation about
 * the mean of the nvec vectors: Xout = mean + inflation (X - mean), the mean
 * in double precision (inflation 1: the exact permutation; in (0, 1000]).
 * The paper's model has its own error growth; a permutation has none, so
 * without inflation a cycled ensemble's spread only shrinks.  X and Xout are
 * distinct.  Any integer shift (taken mod nlon).  Queued on the handle's
 * stream. */
enkfmc_status enkfmc_forecast_shift(enkfmc_handle* h, const void* X, void* Xout, int32_t nvec,
                                    int32_t shift, double inflation);
/* Summand of Eq. 18: *out (device double) = sum_l (mean_m Xa[m][l] - xref[l])^2
 * for Xa [N][n] and xref [n] (device, the handle's element type), the mean and
 * the sum in double precision in a fixed order (the same bits on every run).
 * Queued on the handle's stream. */
enkfmc_status enkfmc_ensemble_sqerr(enkfmc_handle* h, const void* Xa, const void* xref,
                                    double* out);
/* M cycles of Algorithm 1 with enkfmc_forecast_shift (shift, inflation) as the
 * model: for k = 0..M-1,
 * the analysis (enkfmc_estimate, enkfmc_assemble, enkfmc_analyze) of Xb with
 * observations ys[k] ([M][m]) and perturbations Zs[k] ([M][N][m]) into Xa,
 * sqerr[k] = enkfmc_ensemble_sqerr(Xa, xrefs[k]) (xrefs [M][n], the reference
 * states; sqerr device double [M]), then Xb = forecast(Xa).  Eq. 18's RMSE is
 * sqrt(sum_k sqerr[k] / M).  On return Xb holds the forecast after the last
 * analysis and Xa that analysis; Tvals and D the last estimate.  Device
 * buffers, the handle's element type; ys, Zs, Rdiag may be null without
 * observations.  Cycle 0 runs eagerly; the others replay one CUDA graph
 * captured from a private stream (on fixed buffers the handle allocates on the
 * first call; the kernel timing counts the captured cycle once).  Synchronises
 * the handle's stream before the capture and on return.  Numerical failures:
 * enkfmc_get_status. */
enkfmc_status enkfmc_filter_run(enkfmc_handle* h, void* Xb, const void* ys, const void* Zs,
                                const void* Rdiag, const void* xrefs, void* Tvals, void* D,
                                void* Xa, int32_t M, int32_t shift, double inflation,
                                double* sqerr);

/* Reverse pass of the last analysis.  Given Xa_bar = dL/dX^a ([N][n]) of a
 * scalar loss L, writes dL/dy (y_bar, [m]), dL/d diag(R) (Rdiag_bar, [m]) and
 * dL/dX^b (Xb_bar, [N][n]) through every step: the interior write-back
 * (Eq. 10), the sub-domain solves (Eq. 11, with the factors of the last
 * enkfmc_assemble), the assembly of A (Eq. 8), the regressions (Eq. 1-2,
 * Gram factors recomputed from the covariance table, not stored) and the
 * anomalies (Eq. 5).  Requires enkfmc_analyze on this handle, whose inputs
 * (Xb, y, Rdiag, Z) and the Tvals/D of enkfmc_assemble must still hold the
 * same values.  Outputs are overwritten; they may not alias the inputs.
 * Contributions of rows that share predecessors, and of overlapping
 * boundaries, are summed in a fixed order (per component, its blocks in
 * increasing order): the gradients are reproducible bit for bit. */
enkfmc_status enkfmc_analyze_adjoint(enkfmc_handle* h, const void* Xa_bar, void* y_bar,
                                     void* Rdiag_bar, void* Xb_bar);

/* Synchronise the stream; return the first numerical failure recorded since
 * the last call (and clear it).  info (host, nullable) receives the index of
 * the failing row or block. */
enkfmc_status enkfmc_get_status(enkfmc_handle* h, int64_t* info);

/* Number of blocks factored in double precision since the last
 * enkfmc_assemble (single-precision handles; 0 otherwise): those whose
 * single-precision factorisation met a non-positive pivot, and those whose
 * refinement (with three or more steps) converged too slowly after two
 * steps, which enkfmc_analyze moves to double precision for the rest.
 * Synchronises the stream. */
enkfmc_status enkfmc_fp64_blocks(enkfmc_handle* h, int32_t* count /* host */);

/* Strictly-lower pattern of the global T as CSR in label order (host arrays:
 * rowptr [n+1]; colidx [rowptr[n]], or NULL to query the count via
 * rowptr[n]).  Independent of any data. */
enkfmc_status enkfmc_export_T_pattern(const enkfmc_handle* h, int64_t* rowptr, int32_t* colidx);

/* Debug/test access to one block of the factored band after enkfmc_assemble:
 * copies block b's band (column-major lower band, (hb+1) entries per column)
 * into `host` (capacity in elements) and returns nb and hb. */
enkfmc_status enkfmc_debug_block(enkfmc_handle* h, int32_t b, void* host, int64_t capacity,
                                 int64_t* nb, int32_t* hb);

/* Allocation-free estimate.  The paper has no counterpart: this entry point
 * exists for callers that cannot let the library allocate device memory,
 * for example a service that reserves its whole GPU memory budget up front,
 * a host application whose own allocator owns the device, or a
 * latency-critical loop that cannot afford cudaMalloc/cudaFree because they
 * may synchronise the whole device.  It computes the same Tvals [n][pmax] and
 * D [n] as enkfmc_estimate for the problem *p, from Xb [N][n], on
 * `cuda_stream`, without a handle and without allocating anything: its only
 * scratch is one fixed 16 MiB device array inside the library (present on
 * every GPU that loads the library until the process exits).
 *   - Limit: n * (ldN + nC) * sizeof(element) bytes, plus n * (ldN + nC) * 8
 *     for a single-precision problem with rows where 2p > N (2 pmax > N),
 *     each part rounded up to 256 bytes, must fit in 16 MiB (ldN = N rounded
 *     up to a multiple of 4; nC = ((2 vr + 1)(4r + 1)^2 + 1) / 2 pair
 *     covariances per component, vr = min(vert_reach, nlev - 1)).  Larger
 *     problems, and every problem enkfmc_create would refuse as unsupported,
 *     return ENKFMC_EINVAL before anything is queued on the stream.
 *   - The first call on a device looks up the array's device address with
 *     that device current (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - Every call reuses the same array and leaves its contents behind; each
 *     call writes every scratch byte it reads before reading it, so nothing
 *     carries over.  Calls that overlap on the GPU (different streams, or
 *     concurrent host threads) race on the array: serialise them.
 *   - Numerical failures are not reported through a status here: the rows
 *     concerned get D = NaN and a zero T row (test D for NaN).
 * Pointers are device pointers owned by the caller.  Asynchronous. */
enkfmc_status enkfmc_estimate_noalloc(const enkfmc_problem* p, const void* Xb, void* Tvals,
                                      void* D, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batches of independent problems (instances of uneven grid, ensemble size
 * and radius), one CUDA graph per cycle.  The paper analyses independent
 * sub-domains in parallel (Section 3, Algorithm 2); whole instances are
 * independent as well.  A batch keeps references to handles created by the
 * caller (it does not own them; destroy the batch first).  Each instance's
 * estimate -> assemble -> analyze runs on one of `nstreams` side streams,
 * instances placed longest first (by their algorithmic work) on the least
 * loaded stream; enkfmc_batch_capture records the whole fan-out into one
 * graph (captured from a private stream, so `cuda_stream` may be the legacy
 * default stream 0), enkfmc_batch_run launches it on `cuda_stream`.
 * ------------------------------------------------------------------------ */
typedef struct enkfmc_batch enkfmc_batch;

enkfmc_status enkfmc_batch_create(enkfmc_batch** b, enkfmc_handle* const* handles /* host [nprob] */,
                                  int32_t nprob, int32_t nstreams /* 1..64 */, void* cuda_stream);
/* Device buffers of instance i, fixed for the captured graph (layouts as for
 * enkfmc_estimate / _assemble / _analyze; the handle's observations must be
 * set).  Rebinding drops the captured graph. */
enkfmc_status enkfmc_batch_bind(enkfmc_batch* b, int32_t i, const void* Xb, void* Tvals, void* D,
                                const void* y, const void* Rdiag, const void* Z, void* Xa);
/* Synchronises `cuda_stream`, runs one eager cycle of every instance (set-up
 * and numerical status before any replay), then captures one cycle of all of
 * them into a CUDA graph.  Every instance must be bound.  Turns the handles'
 * kernel timing off; on return (success or not) every handle's stream is
 * `cuda_stream` again. */
enkfmc_status enkfmc_batch_capture(enkfmc_batch* b);
/* One cycle of every instance: a single graph launch on the batch's stream. */
enkfmc_status enkfmc_batch_run(enkfmc_batch* b);
/* Synchronise; status[i] (host [nprob]) = instance i's first numerical
 * failure since its last read (enkfmc_get_status), info[i] (host, nullable)
 * its row or block.  Returns the first failing status or OK. */
enkfmc_status enkfmc_batch_get_status(enkfmc_batch* b, int32_t* status, int64_t* info);
/* Side streams and the stream of each instance (host [nprob], nullable). */
enkfmc_status enkfmc_batch_query(const enkfmc_batch* b, int32_t* nstreams, int32_t* stream_of);
void enkfmc_batch_destroy(enkfmc_batch* b);

/* Launch tuning of one handle.  The grid cap is the autotuner's knob and
 * changes no result; the kernel choice changes results at the rounding level
 * (both kernels match the FP64 reference to the single-precision tolerance). */
enum {
  ENKFMC_TUNE_REGRESS_CTAS_PER_SM = 0, /* CTAs per SM of the regressions' grid-stride
                                          launch (0 = the default, 64)              */
  ENKFMC_TUNE_REGRESS_KERNEL = 1       /* single-precision regression kernels:
                                          0 (default) and 1: shared-memory tiled,
                                          a row per warp; 2: register-resident
                                          (forward and adjoint) wherever the
                                          stencil has 16..39 slots; 3: tiled, the
                                          forward rows two per warp (both slower
                                          on the T63 rows)                          */
};
enkfmc_status enkfmc_set_tuning(enkfmc_handle* h, int32_t knob, int32_t value);

/* Kernel kinds launched by the library (index into the profiling arrays). */
enum {
  ENKFMC_K_ANOMALIES = 0,   /* Eq. 5 anomalies, transposed to component-major   */
  ENKFMC_K_REGRESS = 1,     /* Eq. 1-3 regressions of every component            */
  ENKFMC_K_REGRESS_HALO = 2,/* Algorithm 3: boundary rows from local samples     */
  ENKFMC_K_ASSEMBLE = 3,    /* Eq. 11: band of A = T^T D^-1 T + H^T R^-1 H       */
  ENKFMC_K_BANDCHOL = 4,    /* A = L L^T per (sub-domain, variable) block        */
  ENKFMC_K_RHS = 5,         /* H^T R^-1 (Y^s - H X^b)                            */
  ENKFMC_K_BANDSOLVE = 6,   /* L L^T dX = rhs for the N members                  */
  ENKFMC_K_WRITEBACK = 7,   /* Eq. 10 on sub-domain interiors                    */
  ENKFMC_K_COVTABLE = 8,    /* covariances of every pair inside one local box    */
  ENKFMC_K_RESIDUAL = 9,    /* rhs - A dX for the sub-domain refinement step     */
  ENKFMC_K_ADJOINT = 10,    /* reverse pass: seed, observation terms, T Lambda,
                               T dX, anomaly projection                          */
  ENKFMC_K_ADJ_REGRESS = 11,/* reverse pass through the regressions              */
  ENKFMC_K_FP64_BLOCKS = 12,/* single precision: the blocks whose factorisation
                               failed, assembled and factored in double          */
  ENKFMC_K_FORECAST = 13,   /* filter cycling: the forecast operator (advection) */
  ENKFMC_K_SQERR = 14,      /* filter cycling: squared error of the ensemble mean
                               (Eq. 18)                                          */
  ENKFMC_K_DUAL_Z = 15,     /* dual form: Z = T^-T H^T per block (Eq. 13)         */
  ENKFMC_K_DUAL_OBS = 16,   /* dual form: (R + Z^T D Z) W = Y^s - H X^b (Eq. 12)  */
  ENKFMC_K_DUAL_APPLY = 17, /* dual form: dX = T^-1 D Z W (Eq. 12)               */
  ENKFMC_NKERNEL = 18
};

/* Kernel timing.  Work is launched in calls of one kernel kind; a call runs
 * one or more CUDA kernels (the FP32 and FP64 rows of the regressions, the
 * two passes of the refinement residual).  While enabled, every call is
 * bracketed by CUDA events recorded on the handle's stream (the stream its
 * kernels run on).  enkfmc_profile_read synchronises and returns, per kind,
 * the calls and the kernels since the previous read (counted whether or not
 * timing is enabled) and the device time (ms) summed while enabled, then
 * resets.  calls, kernels, ms: host arrays of ENKFMC_NKERNEL. */
enkfmc_status enkfmc_profile(enkfmc_handle* h, int32_t enable);
enkfmc_status enkfmc_profile_read(enkfmc_handle* h, int64_t* calls, int64_t* kernels,
                                  double* ms);
const char* enkfmc_kernel_name(int32_t kind);

/* Algorithmic work of one call of each kernel kind for this problem:
 * floating-point operations of the method (a multiply-add counts 2) and the
 * bytes a kernel must move to or from memory at least (inputs read once,
 * outputs written once).  Implementation extras (refinement passes, re-reads)
 * are not counted.  flops, bytes: host arrays of ENKFMC_NKERNEL.  Entries that
 * depend on the observations are valid after enkfmc_set_observations; those
 * of the dual kinds (ENKFMC_K_DUAL_*) after the first enkfmc_analyze_dual for
 * the current observations. */
enkfmc_status enkfmc_work_per_launch(const enkfmc_handle* h, double* flops, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* ENKFMC_H */
