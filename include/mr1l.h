/*
 * mr1l.h - C ABI of the GB300 multiple rank-1 lattice sparse FFT library.
 *
 * Operations follow Kaemmerer, Potts, Volkmer, "High-dimensional sparse FFT
 * based on sampling along multiple rank-1 lattices":
 *   - a rank-1 lattice Lambda(z, M) = { j z / M mod 1 : j = 0..M-1 } and the
 *     multiple rank-1 lattice (union of L of them), Section 2.1;
 *   - Algorithm 1 (randomized construction, prime set of Eq. 2.2);
 *   - Algorithm 2 (inverse multiple rank-1 lattice FFT, "reconstruct");
 *   - lattice evaluation of a trigonometric polynomial (the aliasing
 *     derivation of Section 4.1) and the adjoint of Algorithm 2;
 *   - Algorithm 3 (dimension-incremental sparse FFT, "sfft_dimincr").
 *
 * Conventions
 *   - Every function returns an int status (MR1L_OK = 0 on success).  No C++
 *     exception crosses this boundary.  mr1l_last_error() copies a message
 *     describing the last failure of the calling thread.
 *   - Complex numbers are interleaved fp64 pairs (re, im), 16 bytes each; the
 *     arrays must be 16-byte aligned.
 *   - "device" pointers are CUDA global memory of the current device, owned
 *     by the caller; "host" pointers are ordinary host memory, owned by the
 *     caller and only read during the call.  A plan owns its own device
 *     buffers and frees them in mr1l_destroy().  Freed library buffers go to
 *     a per-device cache of blocks that later plans and calls reuse (at most
 *     8 GiB kept; freeing synchronises the device, as cudaFree does).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Transforms are asynchronous on that stream; plan creation
 *     and sfft_dimincr synchronise it.
 *   - Lattice sample vectors are stored per lattice: lattice l occupies
 *     positions [off_l, off_l + M_l) with off_l = M_0 + .. + M_{l-1}, node j
 *     of lattice l at off_l + j.  Node 0 (x = 0) belongs to every lattice and
 *     is stored once per lattice.  With nrhs right-hand sides the vectors are
 *     stacked: rhs h starts at h * sum_l M_l.
 *   - Frequencies are rows of int32 (row-major [n][t]).
 *
 * Every routine fails with MR1L_E_INVAL on invalid arguments, MR1L_E_NOMEM
 * when a device allocation fails and MR1L_E_CUDA when a CUDA call or kernel
 * reports an error; the message names the cause.
 */
#ifndef MR1L_H
#define MR1L_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (mr1l_last_error gives the message of the calling thread's
 * last failure) */
#define MR1L_OK 0
#define MR1L_E_INVAL 1              /* invalid argument or unsupported size */
#define MR1L_E_NOMEM 2              /* device or host allocation failed */
#define MR1L_E_CUDA 3               /* a CUDA call or kernel launch failed */
#define MR1L_E_NOT_RECONSTRUCTING 4 /* MR1L_STRICT: some candidate is in no I_l */
#define MR1L_E_SAMPLER 5            /* a user sampler callback returned non-zero */
#define MR1L_E_TIMEOUT 6            /* reserved: no kernel of the library waits on a flag or
                                       on another CTA, so none can time out */

/* plan flags */
#define MR1L_STRICT 1           /* fail with E_NOT_RECONSTRUCTING unless condition (2.1) holds */
#define MR1L_FFT_DF 2           /* Bluestein FFT butterflies in double-float arithmetic (pairs of
                                   FP32 numbers, about 48 significant bits, error-free
                                   transformations) on the FP32 pipes instead of FP64; inputs,
                                   outputs, chirps, the gather and all decisions stay FP64.
                                   Requires |values| between about 1e-30 and 1e30. */
#define MR1L_REDRAW 4           /* mr1l_plan_search: the redraw rule of the original construction
                                   (the remark after Algorithm 1): a lattice whose I_L holds no
                                   frequency the earlier lattices leave uncovered gets a new z_L
                                   (Philox counter word attempt + r 2^16 for the r-th new draw),
                                   at most 64 times, after which the last draw is kept */

/* evaluation modes */
#define MR1L_EVAL 0
#define MR1L_ADJOINT 1

/* threshold modes of sfft_dimincr */
#define SFFT_THETA_ABS 0        /* keep |p~| >= theta (the paper's absolute delta) */
#define SFFT_THETA_REL 1        /* keep |p~| >= theta * max |p~| of the pass */

typedef struct mr1l_plan_s mr1l_plan_t;

/* Copies a NUL-terminated description of the calling thread's last error into
 * buf (at most len bytes).  Returns the status code of that error. */
int mr1l_last_error(char* buf, size_t len);

/* Library version (major * 10000 + minor * 100 + patch). */
int mr1l_version(void);

/* mr1l_pool_stats - the library's cache of device blocks on `device` (every
 * device buffer of plans and solves comes from it): bytes handed out and not
 * yet released (outstanding), bytes of released blocks kept for reuse
 * (cached) and the number of successful cudaMalloc calls so far (mallocs).
 * Any output may be NULL; a device the library has not used reports zeros.
 * Host only.  The paper has no counterpart. */
int mr1l_pool_stats(int device, int64_t* outstanding, int64_t* cached, int64_t* mallocs);

/* mr1l_inject_alloc_failure - a test aid for the error paths: the library's
 * device allocation request that comes `after` requests from now (0 = the
 * next one) fails with MR1L_E_NOMEM, as if the device had run out of memory;
 * -1 cancels a pending injection.  Only the library's host-side allocator is
 * affected; nothing runs on a GPU.  The paper has no counterpart. */
int mr1l_inject_alloc_failure(int64_t after);

/*
 * mr1l_plan - plan the transforms on a given multiple rank-1 lattice.
 * Section 2.1 (lattices, reconstruction property), Algorithm 2 (I_l, counter).
 *   I     host int32 [nI][t]: the frequency set, pairwise distinct, |k_j| < 2^15.
 *   L     number of rank-1 lattices, 1 <= L <= 64.
 *   M     host int64 [L]: lattice sizes, pairwise distinct primes, 2 <= M_l < 2^31.
 *   z     host int64 [L][t]: generating vectors with 0 <= z < M_l.
 *   flags MR1L_STRICT: fail with MR1L_E_NOT_RECONSTRUCTING (and no plan) when
 *         some k in I lies in no I_l.  Without it such k get coefficient 0.
 * Computes the residues k.z_l mod M_l, the collision-free sets I_l and the
 * per-frequency counters on the GPU, and the Bluestein chirp and filter tables
 * of every lattice.  *out receives the plan; destroy it with mr1l_destroy.
 */
int mr1l_plan(const int32_t* I, int64_t nI, int t, int L, const int64_t* M, const int64_t* z,
              int flags, void* stream, mr1l_plan_t** out);

/*
 * mr1l_plan_search - build the lattice by Algorithm 1 (c, gamma), repeated up
 * to b times until condition (2.1) holds (step 2b of Algorithm 3).  The prime
 * sizes are the Lmax smallest primes above lambda = c (|I| - 1) on which
 * k -> k mod p is injective (Eq. 2.2); z_l is drawn uniformly from
 * [1, M_l - 1]^t as 1 + (u mod (M_l - 1)), u the first 64-bit word of
 * Philox4x32-10 with key = seed and counter (j, l, attempt, 3 << 24 | t).
 * When all b searches fail the last one is kept (flags MR1L_STRICT turns that
 * into MR1L_E_NOT_RECONSTRUCTING).
 */
int mr1l_plan_search(const int32_t* I, int64_t nI, int t, double c, double gamma, int b,
                     uint64_t seed, int flags, void* stream, mr1l_plan_t** out);

/*
 * mr1l_plan_info - L, the lattice sizes (M_out: host int64 [64], may be NULL),
 * generating vectors (z_out: host int64 [L][t], may be NULL), the node count
 * 1 - L + sum M_l, the total sample-vector length sum M_l and the number of
 * frequencies that no lattice covers.  Any output pointer may be NULL.
 */
int mr1l_plan_info(const mr1l_plan_t* plan, int* L, int64_t* M_out, int64_t* z_out,
                   int64_t* nodes, int64_t* sum_M, int64_t* n_uncovered);

/* mr1l_plan_masks - the collision-free sets as bitmasks (host uint64 [nI]:
 * bit l set iff k in I_l) and, optionally, the residues (host uint32 [L][nI]). */
int mr1l_plan_masks(const mr1l_plan_t* plan, uint64_t* masks, uint32_t* residues);

void mr1l_destroy(mr1l_plan_t* plan);

/*
 * mr1l_reconstruct - Algorithm 2 on the GPU.
 *   y  device complex [nrhs][sum_l M_l]: samples p(j z_l / M_l mod 1).
 *   c  device complex [nrhs][nI]: p~_k = (1/counter_k) sum_{l: k in I_l}
 *      (1/M_l) sum_j y_{l,j} exp(-2 pi i j k.z_l / M_l);  0 where counter_k = 0.
 * Each length-M_l DFT runs as a Bluestein convolution over FFTs of length 2^k
 * or 3 * 2^k (the smallest such P >= 2 M_l - 1), in FP64 or, with the plan
 * flag MR1L_FFT_DF, in double-float butterflies; the gather of the averaged
 * coefficients is fused with the final chirp.
 */
int mr1l_reconstruct(mr1l_plan_t* plan, const void* y, int nrhs, void* c, void* stream);

/*
 * mr1l_evaluate - lattice evaluation and the adjoint of Algorithm 2.
 *   c  device complex [nrhs][nI], y device complex [nrhs][sum_l M_l].
 *   MR1L_EVAL:    y_{l,j} = sum_{k in I} c_k exp(2 pi i j k.z_l / M_l)
 *                 (the polynomial sum_k c_k e^{2 pi i k.x} at the nodes);
 *   MR1L_ADJOINT: y_{l,j} = sum_{k in I_l} c_k / (counter_k M_l) exp(2 pi i j k.z_l / M_l)
 *                 (the conjugate transpose of mr1l_reconstruct).
 * Both are an inverse Bluestein transform of lattice bins.  EVAL sums the
 * coefficients into bins k.z_l mod M_l with atomics (colliding frequencies
 * share a bin).  ADJOINT writes every bin once from a bin -> frequency map
 * that the plan builds on its first adjoint (sum_l M_l int32 and nI doubles
 * of device memory, kept with the plan, plus nrhs x nI complex scratch for
 * the scaled coefficients); its 1/M_l is applied after the transform.
 */
int mr1l_evaluate(mr1l_plan_t* plan, const void* c, int nrhs, void* y, int mode, void* stream);

/*
 * mr1l_reconstruct_batch / mr1l_evaluate_batch - the transforms of `count`
 * plans in one call: entry i is mr1l_reconstruct(plans[i], y[i], nrhs[i],
 * c[i]) (or mr1l_evaluate(plans[i], c[i], nrhs[i], y[i], mode)).  The entries
 * run on up to 8 internal streams forked from `stream` and joined back into
 * it, so work queued on `stream` before the call comes first and work queued
 * after it sees every result.  Entries naming the same plan run in order on
 * one internal stream (a plan's scratch serves one transform at a time).  The
 * call fails on the first invalid entry; entries before it may have been
 * queued.  The paper has no counterpart: it batches independent transforms.
 */
int mr1l_reconstruct_batch(mr1l_plan_t* const* plans, int count, const void* const* y, const int* nrhs,
                           void* const* c, void* stream);
int mr1l_evaluate_batch(mr1l_plan_t* const* plans, int count, const void* const* c, const int* nrhs,
                        void* const* y, int mode, void* stream);

/*
 * mr1l_reconstruct_noalloc - the same result as mr1l_reconstruct without any
 * device allocation (the paper has no counterpart; this serves callers that
 * cannot allocate device memory while they run: hosts whose device memory is
 * owned entirely by another allocator or budget, and latency-critical loops
 * that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * cause).  The caller still passes y and c exactly as for mr1l_reconstruct;
 * the intermediate FFT data lives in one fixed scratch array compiled into
 * the library (32 MiB per GPU that loads it, held until the process exits).
 *   - Fails with MR1L_E_INVAL, naming both numbers, when nrhs * (sum_l M_l +
 *     L * P) exceeds the fixed maximum of 2^21 complex elements (P is the
 *     plan's Bluestein length, the smallest 2^k or 3 * 2^k >= 2 max M_l - 1).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.  With CUDA's default
 *     lazy module loading, that first call may also load the library's device
 *     code on the device and commit the array's 32 MiB there; later calls
 *     allocate nothing.
 *   - Every call shares the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and must be serialised by the
 *     caller.  No part of the array needs to start at zero.
 *   - Allocates nothing on the device and calls no allocating routine (with
 *     kernel profiling, mr1l_prof_enable, left off).
 */
int mr1l_reconstruct_noalloc(mr1l_plan_t* plan, const void* y, int nrhs, void* c, void* stream);

/* ------------------------------------------------------------------------ */
/* Algorithm 3                                                               */
/* ------------------------------------------------------------------------ */

#define SFFT_REQ_LINE 0
#define SFFT_REQ_LATTICE 1

/* A request for samples of the black-box function p (Algorithm 3, steps 1,
 * 2a and 2c-2d).  Anchors are the random components x' (all d entries are
 * given; the entries the nodes replace are ignored).
 *   LINE:    nodes (x'_1, .., x'_{t-1}, l / K, x'_{t+1}, .., x'_d), l = 0..K-1;
 *            y receives K values.
 *   LATTICE: nodes (j z_l / M_l mod 1, x'_{t+1}, .., x'_d) for every lattice l
 *            and j = 0..M_l - 1, stored per lattice as above (sum M_l values).
 * y is a device pointer into library memory, valid during the callback; the
 * callback must enqueue its work on `stream` (or finish it before returning). */
typedef struct sfft_request {
    int kind;               /* SFFT_REQ_LINE or SFFT_REQ_LATTICE */
    int t;                  /* 1-based dimension increment */
    int rep;                /* 0-based detection iteration */
    int d;
    const double* anchors;  /* host double [d] */
    int K;                  /* LINE: number of nodes */
    int L;                  /* LATTICE: lattices, sizes and generating vectors */
    const int64_t* M;       /* host int64 [L] */
    const int64_t* z;       /* host int64 [L][t] */
    int64_t sum_M;
} sfft_request;

typedef int (*sfft_sample_fn)(void* user, const sfft_request* req, void* y, void* stream);

#define SFFT_SAMPLER_PLANTED 0
#define SFFT_SAMPLER_BSPLINE 1

/* Sampler: either a user callback, or (fn == NULL) a built-in one:
 *
 * SFFT_SAMPLER_PLANTED (kind 0): the planted sparse polynomial
 * p(x) = sum_h c_h e^{2 pi i h.x} plus complex Gaussian noise
 * eta = sigma/sqrt(2) (g1 + i g2) (Section 5.2), drawn with Philox purposes 4
 * and 5 keyed by noise_seed.  It evaluates lattices by the Section 4.1
 * aliasing identity (bin h_(1..t).z_l mod M_l, weight c_h e^{2 pi i h_(>t).x'})
 * and an inverse Bluestein DFT.
 *
 * SFFT_SAMPLER_BSPLINE (kind 1): the tensor-product B-spline function of
 * Section 5.3, f(x) = sum_g prod_{t: group_of[t] = g} N_{orders[g]}(x_t),
 * N_m(x) = C_m sum_k sinc(pi k/m)^m (-1)^k e^{2 pi i k x} with ||N_m|| = 1,
 * evaluated at every node in the spatial domain (N_m(x) = C_m m B_m(m x) with
 * the cardinal B-spline B_m); noiseless (sigma must be 0), freqs/coeffs unused,
 * orders in [2, 8], at most 8 groups, d <= 64. */
typedef struct sfft_sampler {
    sfft_sample_fn fn;
    void* user;
    const int32_t* freqs;   /* planted: host int32 [s][d] */
    const double* coeffs;   /* planted: host complex [s] */
    int64_t s;
    double sigma;
    uint64_t noise_seed;
    int device_arrays;      /* planted: 1 if freqs and coeffs are device pointers */
    int kind;               /* fn == NULL: SFFT_SAMPLER_PLANTED (0) or SFFT_SAMPLER_BSPLINE */
    int n_groups;           /* bspline: number of tensor-product terms */
    const int* group_of;    /* bspline: host int [d]: term of each dimension, or -1 (absent) */
    const int* orders;      /* bspline: host int [n_groups]: B-spline order of each term */
} sfft_sampler;

typedef struct sfft_params {
    int d;                  /* dimension, >= 2 */
    int N;                  /* search domain Gamma = {-N..N}^d, 1 <= N <= 2048 */
    int64_t s;              /* sparsity parameter (final cap) */
    int64_t s_local;        /* per-pass cap for t < d (paper default: s) */
    int r;                  /* detection iterations */
    int b;                  /* lattice searches per increment (total) */
    double theta;           /* threshold */
    int theta_mode;         /* SFFT_THETA_ABS or SFFT_THETA_REL */
    uint64_t seed;          /* Philox key of anchors and generating vectors */
    int batch_reps;         /* 0: one repetition per launch sequence; 1: all r~ fused */
    int fft_arith;          /* 0: FP64 Bluestein FFTs; 1: double-float (see MR1L_FFT_DF) */
    int t_stop;             /* 0: all d increments; 2 <= t_stop < d: stop after increment t_stop
                               and return the projected set I^(1..t_stop) (rows of t_stop
                               components, coefficients zero) - a bounded prefix of the run */
    int zero_anchors;       /* 1: the anchor components x'_1..x'_d of every line and lattice
                               pass are 0 instead of Philox draws - the deterministic variant
                               the paper remarks on in Section 3 for coefficients whose real
                               parts (or imaginary parts) all share one sign, meant for r = 1;
                               the lattices are still drawn (Algorithm 1) */
    int redraw;             /* 1: Algorithm 1 with the redraw rule of the remark after it (see
                               MR1L_REDRAW); 0: Algorithm 1 as printed */
} sfft_params;

#define SFFT_MAX_STEPS 256

typedef struct sfft_step_stats {
    int t;
    int n_line;             /* |I^(t)| */
    int64_t n_cand;         /* |J_t| */
    int L;
    int attempts;
    int covered;
    int64_t sum_M;
    int64_t samples;        /* samples requested at this increment */
    int64_t n_detected;     /* |I^(1..t)| */
} sfft_step_stats;

typedef struct sfft_stats {
    int n_steps;
    int64_t samples;        /* total samples, distinct nodes counted once */
    double ms_total;
    double ms_sampling;     /* time inside the sampler (GPU events) */
    sfft_step_stats steps[SFFT_MAX_STEPS];
} sfft_stats;

typedef struct sfft_result {
    int64_t n;              /* detected frequencies */
    int d;
    int32_t* freqs;         /* host int32 [n][d], lexicographic */
    double* coeffs;         /* host complex [n] */
    sfft_stats stats;
} sfft_result;

/*
 * sfft_dimincr - Algorithm 3 on the GPU.  The detected set and its
 * coefficients (those of the single pass at t = d) are returned in a result
 * owned by the library; release it with sfft_free.  Within one call the
 * Bluestein filter spectrum of a lattice size is computed once and reused by
 * later increments with the same size and Bluestein length (up to 2 GiB of
 * spectra; the environment variable MR1L_FILTER_CACHE=0 turns this off; the
 * results are the same bit for bit either way).
 */
int sfft_dimincr(const sfft_params* params, const sfft_sampler* sampler, void* stream,
                 sfft_result** out);

void sfft_free(sfft_result* res);

/*
 * sfft_select - the thresholded "(up to) s-largest" selection of Algorithm 3
 * (steps 1, 2a and 2e) on its own, over nrhs segments of n values each.
 *   p        device complex [nrhs][n]: the values p~_k of one pass per segment.
 *   eligible device uint8 [n] or NULL: 0 marks an index that is never selected
 *            (a candidate no lattice covers); NULL: all eligible.
 *   cap      keep at most cap indices per segment (0: none).
 *   theta    threshold: key >= theta^2 (SFFT_THETA_ABS) or key >= theta^2 times
 *            the segment's largest eligible key (SFFT_THETA_REL), with key =
 *            re*re + im*im rounded per operation (no fused multiply-add).
 *   flags    device uint8 [n]: set to 1 at every index some segment selects
 *            (the union over segments, as Algorithm 3 unites its passes);
 *            entries not selected are left as they are.
 * Within a segment the largest keys win and equal keys go to the smaller
 * index.  Asynchronous on `stream`; its scratch comes from the block cache,
 * whose release synchronises the device.
 */
int sfft_select(const void* p, int64_t n, int nrhs, const uint8_t* eligible, int64_t cap, double theta,
                int theta_mode, uint8_t* flags, void* stream);

/*
 * sfft_theorem_params - the parameters of the theorem in Section 4 that
 * bounds the failure probability of Algorithm 3 by eps (0 < eps < 1) for a
 * polynomial with `supp` non-zero coefficients in d dimensions:
 *   r = ceil(2 supp (ln 3 + ln d + ln supp - ln eps))   detection iterations,
 *   b = ceil((ln 3 + ln d - ln eps) / ln 2)            lattice searches.
 * (Natural logarithms.)  The theorem also asks for an absolute threshold
 * delta <= min |c| / 3 and s >= supp.  These r are far above what the
 * experiments need (r = 1..5), so they are a worst-case setting.  Host only.
 * Returns MR1L_E_INVAL for d < 1, supp < 1 or eps outside (0, 1).
 */
int sfft_theorem_params(int d, int64_t supp, double eps, int64_t* r, int* b);

/*
 * sfft_dimincr_batch - Algorithm 3 on `count` independent problems
 * (params[i], samplers[i]; uneven d, N, s allowed).  Up to `concurrency`
 * problems run at once, each on its own non-blocking CUDA stream driven by its
 * own host worker, so the small launches of one problem overlap the work of
 * the others.  out[i] receives problem i's result (free each with sfft_free)
 * and status[i] its status; the call returns the first failure's status (the
 * other problems still run).  Host arrays of every sampler must stay valid
 * for the whole call.
 */
int sfft_dimincr_batch(const sfft_params* params, const sfft_sampler* samplers, int count, int concurrency,
                       sfft_result** out, int* status);

/*
 * mr1l_lattice_noise - the measurement noise of the built-in planted sampler
 * (Section 5.2): y[off_l + j] = sigma/sqrt(2) (g1 + i g2) for every lattice l
 * (sizes M, host int64 [L]) and node j, by Box-Muller on the Philox4x32-10
 * words with key = seed and counter (j, l or 0 for node 0, rep, 5 << 24 | t).
 * y: device complex [sum M].  Synchronises the stream.
 */
int mr1l_lattice_noise(uint64_t seed, int t, int rep, int L, const int64_t* M, double sigma, void* y,
                       void* stream);

/* ------------------------------------------------------------------------ */
/* Launch accounting and kernel timing                                       */
/* ------------------------------------------------------------------------ */

/* Every kernel launch of the library is counted.  With profiling enabled,
 * each launch is also bracketed by CUDA events on its own stream together
 * with its algorithmic flops and bytes (FFT flops by the 5 n log2 n
 * convention).  mr1l_prof_read writes a JSON object
 *   {"kernel": {"launches": n, "ms": total, "flops": f, "bytes": b}, ...}
 * into buf (len bytes), synchronising the recorded events; it fails with
 * MR1L_E_INVAL when buf is too small. */
int mr1l_prof_enable(int on);
int mr1l_prof_reset(void);
long long mr1l_prof_launches(void);
int mr1l_prof_read(char* buf, size_t len);

/* ------------------------------------------------------------------------ */
/* Tile tuner                                                                */
/* ------------------------------------------------------------------------ */

/* The column and row passes of a Bluestein convolution with P > 4096 run in
 * tiles of 1024, 2048 or 4096 complex elements per CTA.  The first such
 * transform of each (device, P, mode, arithmetic) in the process runs its
 * passes once with the default tiles and once per distinct tiling, timed with
 * CUDA events on the caller's stream (which it synchronises once), and keeps
 * the fastest column and row tiles; the output is the same bit for bit under
 * every tiling.  No trials
 * run while the stream is being captured, under mr1l_reconstruct_noalloc, or
 * when tuning is disabled (mr1l_tune_enable(0), or the environment variable
 * MR1L_TILE_TUNE=0): those transforms use 2048 unless a choice is cached.
 * MR1L_TILES=<col>,<row> (two of 1024, 2048, 4096) fixes the tiles of every
 * transform instead (no trials, nothing cached).
 * The paper has no counterpart (it concerns the GPU implementation only).
 * mr1l_tune_reset forgets every choice; mr1l_tune_read writes the choices as
 * a JSON array of {"device", "P", "mode", "df", "col_tile", "row_tile",
 * "col_ms", "row_ms"} into buf (len bytes; MR1L_E_INVAL when too small). */
int mr1l_tune_enable(int on);
int mr1l_tune_reset(void);
int mr1l_tune_read(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* MR1L_H */
