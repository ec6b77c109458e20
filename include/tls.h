/*
 * tls.h -- C ABI of the GB300 two-link staggered quark smearing library.
 *
 * The method (Gottlieb, Jeong, Strelchenko, arXiv:2301.05518, Sec. 2-3):
 *
 *   two-link product    W_i(x) = U_i(x) U_i(x + i),  i = x, y, z
 *                       (Sec. 2, the definition before Eq. tlLapl1)
 *   two-link Laplacian  Delta psi(x) = 4 Lap_two psi(x)
 *                         = sum_i [ W_i(x) psi(x + 2i) + W_i^dag(x - 2i) psi(x - 2i) ]
 *                           - 6 psi(x)                     (Sec. 2, Eq. tlLapl1)
 *   smearing            psi <- (1 + (sigma/N) Lap_two)^N psi   (Sec. 2, Eq. tlSmear)
 *                       = N steps of psi <- psi + (sigma / (4N)) Delta psi
 *   reuse               W is computed once per gauge field and reused for
 *                       every iteration, source and sink     (Sec. 3)
 *
 * Every entry point returns a tls_status: TLS_OK (0) or a negative code.  No
 * entry point aborts or throws across the ABI.  tls_last_error() gives a
 * message for the last failing call on the calling thread.
 *
 * Layouts seen by the caller (all "canonical", x fastest):
 *   gauge links U : double [Lt][Lz][Ly][Lx][nd][3][3][2], nd = 3 (mu = x, y, z)
 *                   or 4 (mu = x, y, z, t; the t links are ignored)
 *   vectors       : [nvec][Lt][Lz][Ly][Lx][3][2] of double (TLS_F64) or float
 *                   (TLS_F32); a colour vector of 3 complex numbers per site.
 * dims[4] = {Lx, Ly, Lz, Lt}.  Every spatial extent must be even (the +-2
 * hops must keep the 8 spatial-parity sublattices apart, Sec. 2: the operator
 * preserves taste); Lt >= 1.  Boundaries are periodic in x, y, z; t is never
 * shifted, every time slice is an independent problem.
 *
 * Threads: one tls_ctx may be used from several host threads; calls on one
 * context are serialised internally.  Streams: a NULL stream means the CUDA
 * legacy default stream of the context's device.
 */
#ifndef TLS_H
#define TLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tls_ctx tls_ctx;
typedef int64_t tls_gauge_id;
typedef int tls_status;

/* ---- status codes ------------------------------------------------------- */
#define TLS_OK               0
#define TLS_ERR_ARG         -1  /* invalid argument (odd extent, N < 0, ...)  */
#define TLS_ERR_NOMEM       -2  /* cudaMalloc failed                          */
#define TLS_ERR_ADMIT       -3  /* would exceed the context's HBM cap         */
#define TLS_ERR_CUDA        -4  /* a CUDA runtime call failed                 */
#define TLS_ERR_TIMEOUT     -5  /* a bounded device wait ran out              */
#define TLS_ERR_NOT_BUILT   -6  /* smear requested before tls_build_twolink   */
#define TLS_ERR_DEVICE      -7  /* the device error word was set by a kernel  */
#define TLS_ERR_STATE       -8  /* call not valid in the current state        */
#define TLS_ERR_UNSUPPORTED -9  /* precision / recon / kernel combination     */
#define TLS_ERR_NOT_FOUND  -10  /* unknown gauge id or job id                 */

/* ---- precisions (storage and I/O) ---------------------------------------- */
#define TLS_F64  0
#define TLS_F32  1
#define TLS_F16  2  /* 16-bit storage with one FP32 scale per site and vector */
#define TLS_BF16 3

/* ---- W compression: reals stored per 3x3 complex matrix ------------------ */
#define TLS_R18 18  /* all 9 complex entries                                  */
#define TLS_R12 12  /* rows 1-2; row 3 = conj(row1 x row2) (W is SU(3))       */
#define TLS_R8   8  /* W01, W02, W10, arg W00, arg W20; needs |W00| < 1       */

/* ---- kernel choice for tls_smear ----------------------------------------- */
#define TLS_KERNEL_AUTO       0  /* planner / autotune table decides          */
#define TLS_KERNEL_SINGLE     1  /* one vector per launch, one launch per step */
#define TLS_KERNEL_MRHS       2  /* all vectors in one launch: W read once     */
#define TLS_KERNEL_PERSISTENT 3  /* all N steps in one cooperative launch,     */
                                 /* tiles kept L2-resident between steps       */
#define TLS_KERNEL_MRHS_ROWS  4  /* multi-RHS, rows staged in shared memory by */
                                 /* TMA bulk copies (falls back to MRHS when   */
                                 /* the shape does not allow 16-byte copies)   */
#define TLS_KERNEL_MRHS_ZM    5  /* multi-RHS, each thread marches along z     */
                                 /* with the z-neighbours in registers         */

#define TLS_ALL_T (-1)           /* timeslice argument: smear every slice      */

/* ---- context -------------------------------------------------------------
 * tls_create: a context on CUDA device `device`.  hbm_cap_bytes bounds the
 * device memory the context may hold (gauge fields, two-link fields, vector
 * workspaces, serving slots); 0 means no cap.  *out is NULL on failure.
 * tls_destroy frees everything the context owns (stops serving first).   */
tls_status tls_create(tls_ctx **out, int device, uint64_t hbm_cap_bytes);
void tls_destroy(tls_ctx *ctx);

/* Message of the last failing tls_* call on this host thread ("" if none).
 * The pointer stays valid until the next tls_* call on the same thread.   */
const char *tls_last_error(void);

/* Library version, e.g. 10000 for 1.0.0. */
int tls_version(void);

/* Device bytes currently held by the context. */
uint64_t tls_bytes_in_use(const tls_ctx *ctx);

/* ---- gauge field ingest (Sec. 2: U_mu(x)) ----------------------------------
 * Copies the spatial links of U (layout above, FP64) to the device and
 * permutes them into the library's sublattice layout (bit-exact).  U is a
 * device pointer if on_device != 0, else a host pointer (only the spatial
 * links are copied, in slice groups whose copy overlaps the permutation of
 * the previous group); the caller keeps ownership and may free it when the
 * call returns.  The work is enqueued on
 * `stream` and finished before return.  Returns the new id in *out.
 * Errors: TLS_ERR_ARG (nd not 3/4, odd or non-positive extent, more than
 * 2^31 sites), TLS_ERR_ADMIT, TLS_ERR_NOMEM, TLS_ERR_CUDA.                  */
tls_status tls_load_gauge(tls_ctx *ctx, const double *U, int nd, const int dims[4],
                          int on_device, void *stream, tls_gauge_id *out);

/* ---- two-link build (Sec. 2 definition of V_mu; Sec. 3 precompute) ---------
 * W_i(x) = U_i(x) U_i(x+i) for every site and i = x, y, z, formed in FP64
 * and rounded to nearest in `wprec` (TLS_F64, TLS_F32, TLS_F16, TLS_BF16),
 * stored with `recon` reals per matrix (TLS_R18; TLS_R12 or TLS_R8 for FP32;
 * TLS_R12 for 16-bit).  W stays resident until tls_free_gauge.  keep_U = 0
 * releases the device copy of U after the build.  Rebuilding replaces W.
 * Errors: TLS_ERR_NOT_FOUND, TLS_ERR_STATE (U already released),
 * TLS_ERR_UNSUPPORTED (combination), TLS_ERR_DEVICE (TLS_R8 met a matrix with
 * |W00| too close to 1 to parameterise), memory errors.                     */
tls_status tls_build_twolink(tls_ctx *ctx, tls_gauge_id id, int wprec, int recon,
                             int keep_U, void *stream);

/* ---- one-link field (Sec. 2, Eq. 2: the links U_mu of the hopping term) -----
 * Stores the spatial links U_mu(x) themselves, rounded to nearest in `prec`
 * (TLS_F64 or TLS_F32), in the two-link field's layout, for
 * tls_smear_onelink.  keep_U = 0 releases the FP64 device copy of U.
 * Errors: TLS_ERR_NOT_FOUND, TLS_ERR_STATE (U released), TLS_ERR_UNSUPPORTED. */
tls_status tls_build_links(tls_ctx *ctx, tls_gauge_id id, int prec, int keep_U, void *stream);

/* ---- gauge-smeared links (Sec. 2, the remark after Eq. tlSmear) -------------
 * Replaces the resident FP64 spatial links of gauge `id` by n_steps steps of
 * APE smearing, each computed from the previous links (out of place):
 *     V_mu(x) = (1 - alpha) U_mu(x) + (alpha/4) sum_{nu != mu, spatial} [
 *         U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
 *     U'_mu(x) = P(V_mu(x)),
 * P being the projection onto SU(3): the unitary polar factor (Newton's
 * iteration X <- (X + X^-dag)/2) times exp(-i phi/3), phi = arg det in
 * (-pi, pi].  Staples stay inside each time slice; periodic in x, y, z.  The
 * two-link field and the one-link field built before become invalid
 * (tls_smear then returns TLS_ERR_NOT_BUILT until tls_build_twolink runs
 * again).  Allocates one temporary copy of the links.
 * Errors: TLS_ERR_NOT_FOUND, TLS_ERR_STATE (U released), TLS_ERR_ARG
 * (n_steps < 0 or alpha outside [0, 1]), TLS_ERR_DEVICE (a projection met a
 * singular matrix or did not settle; that link kept its previous value),
 * memory and CUDA errors.                                                     */
tls_status tls_ape_smear(tls_ctx *ctx, tls_gauge_id id, double alpha, int n_steps, void *stream);

/* Releases U, W and everything cached for gauge `id`. */
tls_status tls_free_gauge(tls_ctx *ctx, tls_gauge_id id);

/* Copies W back out in FP64, canonical layout [Lt][Lz][Ly][Lx][3][3][3][2]
 * (i, row, col, re/im), reconstructing compressed forms.  `out` is a host
 * pointer (on_device = 0) or device pointer (on_device != 0) of V*162
 * doubles.  For tests of the build.                                        */
tls_status tls_export_twolink(tls_ctx *ctx, tls_gauge_id id, double *out, int on_device,
                              void *stream);

/* Copies the device copy of the spatial links back out in canonical layout
 * [Lt][Lz][Ly][Lx][3][3][3][2] (bit-exact inverse of the ingest).          */
tls_status tls_export_gauge(tls_ctx *ctx, tls_gauge_id id, double *out, int on_device,
                            void *stream);

/* ---- smearing (Sec. 2, Eq. tlSmear with Eq. tlLapl1) -------------------------
 * Applies psi <- (1 + (width/N) Lap_two)^N psi to each of the nvec vectors in
 * place.  width is the paper's sigma; each step is
 *     psi'(x) = psi(x) + (width/(4N)) Delta psi(x)   (out of place, Jacobi).
 * timeslice in [0, Lt) smears that slice only and leaves the other slices of
 * `vecs` untouched; TLS_ALL_T smears every slice.
 *   vecs            caller's vectors, layout above, io_prec TLS_F64 or TLS_F32;
 *                   device pointer if vecs_on_device != 0, else host pointer:
 *                   then the slices go through the device in groups of about
 *                   2 GB, the copy of one group in, the smearing of another
 *                   and the copy of a third back out overlapping on three
 *                   streams (pinned host memory lets the copies run at full
 *                   speed).
 *   storage         precision the iterates are stored in between steps:
 *                   TLS_F64 (needs an FP64 W), TLS_F32 (FP32 W), TLS_F16 or
 *                   TLS_BF16 (FP32 or 16-bit W; one FP32 scale per site and
 *                   vector; arithmetic in FP32).
 *   kernel          TLS_KERNEL_* above.
 *   norms_out       NULL or a host array of nvec doubles: ||psi_v||^2 of each
 *                   smeared vector over the smeared slices, summed in FP64 in
 *                   a fixed order (deterministic).
 * N = 0 or width = 0 returns the input unchanged in value, up to one rounding
 * to `storage` when it is narrower than io_prec.  Each vector's result is
 * bitwise independent of nvec and of the other vectors for a given (kernel,
 * storage, W format).  The call is synchronous: it returns when the result is
 * in `vecs`.
 * Errors: TLS_ERR_ARG, TLS_ERR_NOT_FOUND, TLS_ERR_NOT_BUILT,
 * TLS_ERR_UNSUPPORTED, TLS_ERR_TIMEOUT (persistent kernel barrier ran out; the
 * vectors are then unspecified), TLS_ERR_DEVICE, memory and CUDA errors.    */
tls_status tls_smear(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec,
                     int vecs_on_device, int nvec, int N, double width, int timeslice,
                     int storage, int kernel, void *stream, double *norms_out);

/* ---- one-link Gaussian smearing (Sec. 2, Eq. 2-3) ---------------------------
 * Applies psi <- C (1 + alpha H)^N psi with C = 1 (Eq. 3), where
 *     H psi(x) = sum_mu [ U_mu(x) psi(x + mu) + U_mu^dag(x - mu) psi(x - mu) ]
 * is the one-link hopping operator of Eq. 2 (mu = x, y, z; periodic), each
 * step psi' = psi + alpha H psi out of place.  The Laplacian form of Eq. 4,
 * C' (1 + alpha' Lap)^N, is the same operator with alpha = alpha'/(1 - 6 alpha')
 * and C' = (1 + 6 alpha)^N.  Needs tls_build_links (FP64 links for TLS_F64
 * storage, FP32 links otherwise).  Vectors, slices, storage, norms and errors
 * as tls_smear (multi-right-hand-side kernel, interleaved layout).          */
tls_status tls_smear_onelink(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int vecs_on_device, int nvec,
                             int N, double alpha, int timeslice, int storage, void *stream, double *norms_out);

/* ---- smearing without any device allocation --------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory while they run: a latency-critical host
 * thread (cudaFree synchronises the whole device), or a process whose device
 * memory belongs to another allocator.
 * It computes what tls_smear(..., kernel = TLS_KERNEL_PERSISTENT, ...) does,
 * on device vectors only (`vecs` is device memory of the context's device,
 * canonical layout, smeared in place), and calls no cudaMalloc, cudaFree or
 * other allocating routine.  All its intermediate data lives in one static
 * device array of TLS_NOALLOC_SCRATCH_BYTES that every device loading the
 * library holds until the process exits; a smear whose packed vectors and
 * persistent-kernel scratch do not fit is rejected with TLS_ERR_ARG (use
 * tls_smear for it).  The first call on a device looks up the array's device
 * address with that device current.  Calls share the array: each clears
 * what must start at zero, and calls whose work overlaps on the GPU race on
 * it.  The gauge must
 * already be built (tls_build_twolink allocates W; this call does not).
 * Synchronous on `stream`: it waits for the stream and copies the device
 * error word into host memory before it returns.  Errors as tls_smear; after
 * TLS_ERR_TIMEOUT or TLS_ERR_DEVICE the vectors are unspecified.           */
#define TLS_NOALLOC_SCRATCH_BYTES (32u << 20)
tls_status tls_smear_noalloc(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int nvec, int N,
                             double width, int timeslice, int storage, void *stream);

/* ---- per-call profile ------------------------------------------------------
 * With profiling on (tls_set_profiling), each tls_smear / tls_build_twolink
 * records CUDA events on its stream around its phases.                     */
typedef struct {
    double ms_total;        /* whole call on its stream                        */
    double ms_h2d;          /* host->device copy of the vectors (host input)   */
    double ms_pack;         /* canonical -> sublattice layout (+ quantise)     */
    double ms_iter;         /* all smearing steps                              */
    double ms_unpack;       /* sublattice -> canonical (+ norms)               */
    double ms_d2h;          /* device->host copy of the vectors (host input)   */
    double ms_build;        /* tls_build_twolink: the build kernel             */
    int64_t launches;       /* kernel launches of the call                     */
    int64_t iter_launches;  /* kernel launches in the iteration phase          */
    double iter_bytes;      /* algorithmic bytes of the iteration phase:
                               W once + psi read once + psi written once per
                               site and step                                   */
    double iter_flops;      /* algorithmic flops of the iteration phase        */
    int kernel;             /* TLS_KERNEL_* that actually ran                  */
    int vecs_per_thread;    /* vectors per thread of the stencil kernel        */
} tls_profile;

tls_status tls_set_profiling(tls_ctx *ctx, int on);
tls_status tls_get_profile(tls_ctx *ctx, tls_profile *out);

/* Testing hook for the bounded device waits of the persistent kernel: the
 * spin budget, in polls, of each inter-block barrier (0 restores the default).
 * A tiny budget forces the TLS_ERR_TIMEOUT path without hanging the GPU.   */
tls_status tls_set_barrier_budget(tls_ctx *ctx, int64_t polls);

/* ---- autotuning ------------------------------------------------------------
 * Candidate kernels for one problem shape, each timed with CUDA events over
 * `steps` smearing steps on scratch vectors of the context's device.        */
typedef struct {
    int kernel;             /* TLS_KERNEL_SINGLE, _MRHS or _PERSISTENT         */
    int vecs_per_thread;    /* vectors per thread (planar kernels)             */
    int threads;            /* threads per CTA                                 */
    int tile[3];            /* multi-RHS kernel: tile[0] > 0 sets the sites    */
                            /* per CTA (a strip along x'); persistent kernel:  */
                            /* tile[0] > 0 sets the L2 budget of one group of  */
                            /* blocks in MB (default 48), tile[1] = 1 selects  */
                            /* the on-chip form (one CTA per block keeps W and */
                            /* the iterates in shared memory, when they fit);  */
                            /* multi-RHS kernel:                               */
                            /* tile[1] = 1 stages the strip's W in shared      */
                            /* memory, tile[1] = 2 as well and applies it with */
                            /* packed FP32 pair FMAs (not FP64), tile[1] = 3   */
                            /* like 2 with all vector loads issued up front,   */
                            /* tile[1] = 4 stages W as stored and applies it   */
                            /* with packed FP32 pair FMAs, tile[1] = 5 is 2    */
                            /* held to 56 registers in CTAs of <= 96 threads;  */
                            /* tile[1] = 6 runs one CTA per whole x'-row with  */
                            /* the row's five W rows copied in by TMA bulk     */
                            /* copies (tile[0] > 0: vectors per CTA), 7 the    */
                            /* same with the next hop's records requested      */
                            /* early, 8 with the row's own records copied in   */
                            /* as well (FP32 and 16-bit storage; other shapes  */
                            /* take tile[1] = 2);                              */
                            /* tile[2] (tile[1] = 6..8): each CTA requests     */
                            /* into L2 the W rows and records of the row       */
                            /* tile[2] planes ahead in launch order; 0 none,   */
                            /* < 0 the distance that keeps about 12 MB of row  */
                            /* data ahead; other kernels ignore it             */
    double ms_per_step;     /* measured time of one smearing step              */
} tls_tune_entry;

/* Times every candidate for smearing nvec vectors of gauge `id` stored in
 * `storage` on `timeslice` (TLS_ALL_T or a slice), keeps the fastest in the
 * context's table (used by TLS_KERNEL_AUTO for that shape) and returns it in
 * *best (nullable).  Up to max_all candidates are written to `all`
 * (nullable) and their number to *n_all (nullable).  The vectors it smears
 * are scratch: caller data is not touched.  Errors as tls_smear.           */
tls_status tls_autotune(tls_ctx *ctx, tls_gauge_id id, int nvec, int storage, int timeslice, int steps,
                        tls_tune_entry *best, tls_tune_entry *all, int max_all, int *n_all);

/* Sets the table entry for a shape by hand (e.g. from a saved autotune).   */
tls_status tls_tune_set(tls_ctx *ctx, tls_gauge_id id, int nvec, int storage, int timeslice,
                        const tls_tune_entry *entry);

/* ---- serving: continuous batching of smearing jobs (Sec. 6 pattern) ---------
 * A scheduler thread keeps each gauge field's W resident, admits jobs while
 * the context's HBM cap allows, packs the vectors of compatible jobs into the
 * slots of one multi-right-hand-side batch per (gauge id, storage), and
 * advances every active slot one step per launch with the slot's own alpha =
 * width/(4N) and remaining step count.  Jobs arriving while others run join
 * at the next step boundary; finished slots retire and are unpacked.
 * A job's result is bitwise the same alone and in any mix.                  */
typedef struct {
    int max_slots;          /* vectors per batch (per gauge, storage); <= 256  */
    int steps_per_launch;   /* steps advanced between admission points (>= 1)  */
    int use_graphs;         /* capture the per-step launches in CUDA graphs    */
    int reserved[5];
} tls_serve_opts;

typedef struct {
    tls_gauge_id gauge;     /* built gauge field                               */
    void *vecs;             /* host or device vectors, canonical layout;       */
                            /* borrowed until tls_serve_wait returns           */
    int vecs_on_device;
    int io_prec;            /* TLS_F64 or TLS_F32                              */
    int nvec;               /* >= 1                                            */
    int N;                  /* smearing steps, >= 0                            */
    double width;           /* sigma                                           */
    int timeslice;          /* slice or TLS_ALL_T                              */
    int storage;            /* TLS_F32, TLS_F16 or TLS_BF16                    */
    int reserved[4];
} tls_job;

typedef struct {
    tls_status status;      /* TLS_OK or the job's error                       */
    double submit_ms;       /* host clock, ms since tls_serve_start            */
    double start_ms;        /* first step on the device (admission)            */
    double done_ms;         /* result in the caller's buffer                   */
} tls_job_result;

tls_status tls_serve_start(tls_ctx *ctx, const tls_serve_opts *opts);
tls_status tls_serve_stop(tls_ctx *ctx);
/* Non-blocking; copies the descriptor.  TLS_ERR_ADMIT if the job can never
 * fit under the HBM cap.                                                   */
tls_status tls_serve_submit(tls_ctx *ctx, const tls_job *job, uint64_t *job_id);
tls_status tls_serve_poll(tls_ctx *ctx, uint64_t job_id, int *done);
/* Blocks until the job finishes or timeout_s passes (TLS_ERR_TIMEOUT), fills
 * *result (nullable) and releases the job record: a later poll or wait on
 * the same id returns TLS_ERR_NOT_FOUND.  Returns the job's own status.     */
tls_status tls_serve_wait(tls_ctx *ctx, uint64_t job_id, double timeout_s,
                          tls_job_result *result);

/* ---- measurement helper: arithmetic rate of the GPU ------------------------
 * Not a step of the method (the paper has no counterpart); it measures the
 * roof that the FP64 kernels (two-link build, APE step) and the FP32 stencil
 * arithmetic are reported against.  Runs a kernel of independent FMA chains
 * (no memory traffic) on `device`, on a stream of its own, calibrated to about
 * 100 ms per launch, and returns in *tflops the best of several CUDA-event
 * timed launches, counting 2 flops per FMA (per lane for the packed pair
 * form).  Allocates nothing.  Errors: TLS_ERR_ARG (unknown kind or NULL
 * tflops), TLS_ERR_CUDA.                                                    */
#define TLS_PEAK_F64   0  /* fma.rn.f64                                      */
#define TLS_PEAK_F32   1  /* fma.rn.f32                                      */
#define TLS_PEAK_F32X2 2  /* fma.rn.f32x2 (two FP32 lanes per instruction)    */
tls_status tls_peak_flops(int device, int kind, double *tflops);

#ifdef __cplusplus
}
#endif

#endif /* TLS_H */
