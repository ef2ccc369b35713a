/*
 * nnqs.h -- C ABI of the GB300 (sm_103a) library for the local-energy hot
 * path of the transformer neural-network quantum state method (arXiv
 * 2306.16705, "NNQS-Transformer").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Bitstrings are packed into W = ceil(N/64) little-endian uint64 words:
 *   qubit j is bit (j % 64) of word (j / 64); a bitstring occupies W
 *   consecutive words.  Qubit 2p is the alpha spin orbital of spatial
 *   orbital p and qubit 2p+1 its beta partner (Sec. 3.3, interleaved
 *   Jordan-Wigner order).  |1> = occupied.  N <= 128.
 * - log psi is stored as two doubles per state: (log|psi|, phase), so
 *   psi = exp(log|psi| + i phase) (Sec. 3.1 writes psi = |psi| e^{i phi}).
 * - Complex outputs are two doubles (Re, Im).
 * - "device" pointers are CUDA device pointers owned by the caller; "host"
 *   pointers are ordinary host memory owned by the caller.  Opaque handles
 *   are owned by the library and released by the matching *_free.
 * - Calls taking a stream enqueue their work on it and return without
 *   waiting, unless their comment says they synchronise.  Argument errors
 *   are returned synchronously; errors the GPU detects (a sample outside the
 *   electron-number sector, a duplicate sample, a full hash table, a
 *   non-finite value) are written to a status word at the start of the
 *   caller's workspace and read with nnqs_workspace_status().
 * - Workspace: every call that needs scratch device memory takes a
 *   caller-allocated device buffer `workspace` of at least the size its
 *   *_workspace_size function returns (256-byte aligned).  The library
 *   itself allocates device memory only for the Hamiltonian's tables, owned
 *   by its handle (nnqs_build_pauli, nnqs_ham_build_ungrouped); the one
 *   static array of nnqs_eloc_sa_noalloc is documented there.
 * - Empty inputs: nnqs_logpsi with n = 0, nnqs_eloc with n_rows = 0 and
 *   nnqs_sample with n_samples = 0 (*n_unique_out = 0) return NNQS_OK
 *   after their argument checks and launch nothing; nnqs_energy_stats and
 *   nnqs_energy_grad reject an empty sample set with NNQS_E_INVAL (the
 *   weighted mean is undefined).
 * - No exception crosses the ABI.  nnqs_last_error() returns a thread-local
 *   message for the last non-OK status returned on this thread.
 */
#ifndef NNQS_H
#define NNQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *nnqs_stream; /* a cudaStream_t; NULL = default stream */

typedef enum {
    NNQS_OK = 0,
    NNQS_E_INVAL = 1,        /* bad argument (null pointer, size, unsupported shape) */
    NNQS_E_NOMEM = 2,        /* host or device allocation failed */
    NNQS_E_CUDA = 3,         /* a CUDA runtime call failed */
    NNQS_E_TABLE_FULL = 4,   /* a bounded hash probe ran out of slots */
    NNQS_E_TIMEOUT = 5,      /* a bounded device wait gave up */
    NNQS_E_SECTOR = 6,       /* a sample breaks the (n_alpha, n_beta) sector */
    NNQS_E_NONFINITE = 7,    /* NaN or Inf met in an input or result */
    NNQS_E_UNSUPPORTED = 8,  /* valid request the library does not implement */
    NNQS_E_DUPLICATE = 9,    /* the sample table holds a bitstring twice */
    NNQS_E_WORKSPACE = 10    /* workspace null, misaligned or too small */
} nnqs_status;

/* nnqs_eloc modes (Sec. 3.4 (4)): NNQS_SA sums over x' in the sample table
 * S only (the paper's sample-aware scheme); NNQS_EXACT sums over every x'
 * with H_{x x'} != 0 structurally (Eq. Eloc as written). */
enum { NNQS_SA = 0, NNQS_EXACT = 1 };

/* Arithmetic of the ansatz: NNQS_FP64 = FP64 everywhere (the plain path);
 * NNQS_MIXED = BF16 operands on tcgen05 tensor cores with FP32 accumulation
 * and FP32 normalisation/softmax; NNQS_FP32 = FP32 CUDA cores;
 * NNQS_BF16X3 = as NNQS_MIXED, but every forward linear layer splits its
 * operands into high and low BF16 parts (x = x_h + x_l, x_h = bf16(x)) and
 * sums three tensor-core products x_h w_h + x_h w_l + x_l w_h, so log psi
 * carries about 16 operand bits instead of 8 (the reverse mode stays BF16);
 * NNQS_FP8 = every forward linear layer of log psi on tcgen05 with E4M3
 * operands (kind::f8f6f4, FP32 accumulation): activations unscaled, each
 * weight row scaled by a power of two that brings its largest entry into
 * (224, 448] and divided out of the accumulator; the reverse mode and the
 * sampler's conditionals use BF16 operands as NNQS_MIXED does.
 * Local-energy ratios, sums and statistics are FP64 in every mode. */
enum { NNQS_FP64 = 0, NNQS_MIXED = 1, NNQS_FP32 = 2, NNQS_BF16X3 = 3, NNQS_FP8 = 4 };

/* nnqs_eloc flags: choice of the sample-aware sweep.  GROUPS walks the
 * X/Y-mask groups for every sample (Alg. 2); PAIRS walks sample pairs and
 * looks the pair's X/Y mask up in a group hash; AUTO picks the cheaper of
 * the two by their pair counts; TERMS walks every Pauli string with its own
 * X/Y mask (the ungrouped layout the grouping of Alg. 1 replaces, Sec. 3.4;
 * needs nnqs_ham_build_ungrouped).  All give the same sum up to the order of
 * floating-point additions. */
enum { NNQS_SWEEP_AUTO = 0, NNQS_SWEEP_GROUPS = 1, NNQS_SWEEP_PAIRS = 2, NNQS_SWEEP_TERMS = 3 };

const char *nnqs_last_error(void);
const char *nnqs_status_string(int status);
const char *nnqs_version(void);

/* Reads the device status word at the head of `workspace` (synchronises
 * `stream` first).  Returns NNQS_OK or the first error a kernel recorded;
 * `bad_index` (host, may be NULL) receives the offending row or -1. */
nnqs_status nnqs_workspace_status(const void *workspace, nnqs_stream stream, int64_t *bad_index);

/* Tracing.  Every kernel launch is counted per kernel family (the kernel's
 * name); with profiling enabled each launch is also bracketed by CUDA
 * events on its stream.  nnqs_profile_read synchronises the device, folds
 * the recorded events into per-family totals and returns the number of
 * families; family `index` (0-based) fills name (host, name_cap bytes),
 * launches and total_ms (host, may be NULL).  Not part of the numerical
 * method: instrumentation for benchmarks and tests. */
void nnqs_profile_enable(int on);
void nnqs_profile_reset(void);
int nnqs_profile_read(int index, char *name, int name_cap, uint64_t *launches, double *total_ms);
/* algorithmic work the launch sites attributed to family `index` since the
 * last reset: floating-point operations and bytes (host outputs) */
int nnqs_profile_work(int index, double *flops, double *bytes);
uint64_t nnqs_launch_count(void); /* kernel launches since the library loaded */

/* Measured pipe throughput for roofline fractions (instrumentation, not
 * part of the method; the paper has no counterpart).  Register-only loop
 * kernels over every SM, timed with CUDA events on `stream` (best of three
 * after a warm-up launch; synchronises):
 *   out[0]  64-bit XOR + popcount tests per second (the mask test of the
 *           sample-aware sweeps of Alg. 2: two 32-bit logic ops, two
 *           popcounts and one add)
 *   out[1]  32-bit integer ALU operations per second (logic op + add)
 *   out[2]  FP64 FMA flops per second (2 per FMA)
 *   out[3]  FP32 FMA flops per second (2 per FMA)
 * sink: device buffer of nnqs_measure_peaks_sink_size() bytes that receives
 * the loops' results (caller-owned, contents meaningless).  Reads and changes
 * no clock or other device setting.  Errors: NNQS_E_INVAL, NNQS_E_WORKSPACE,
 * NNQS_E_CUDA. */
size_t nnqs_measure_peaks_sink_size(void);
nnqs_status nnqs_measure_peaks(double out[4], void *sink, size_t sink_bytes, nnqs_stream stream);

/* ------------------------------------------------------------------ */
/* Hamiltonian: Eq. (eham) -> Jordan-Wigner Pauli strings, Eq. (sham),  */
/* merged, coefficient-folded and grouped by X/Y mask as in Alg. 1 and  */
/* Sec. 3.4 (1).                                                         */
/* ------------------------------------------------------------------ */
typedef struct nnqs_ham nnqs_ham;

/* Builds H = e_core + sum_{pq,s} h[p][q] a+_{ps} a_{qs}
 *          + 1/2 sum_{pqrs,s,t} eri[p][q][r][s] a+_{ps} a+_{rt} a_{st} a_{qs}
 * (Eq. eham in chemist notation, real integrals), maps it by Jordan-Wigner
 * (a+_j = Z_{<j}(X_j - iY_j)/2), merges equal strings, folds
 * coef = Re(c) Re((-i)^{nY}) (Alg. 1), drops |coef| < drop_tol and groups
 * the survivors by their X/Y mask.  Groups are in ascending X/Y-mask order
 * and terms within a group in ascending Y/Z-mask order (most significant
 * word first).
 *   n_spatial   1..64 spatial orbitals (N = 2 n_spatial qubits)
 *   h           host, n*n row-major, symmetric
 *   eri         host, n^4 row-major (pq|rs), 8-fold symmetric
 *   out         receives the handle; its tables are uploaded to the current
 *               CUDA device (the library allocates them with cudaMalloc).
 * Runs on the host (OpenMP) and synchronises the device once. */
nnqs_status nnqs_build_pauli(int n_spatial, const double *h, const double *eri, double e_core,
                             double drop_tol, nnqs_ham **out);

/* nnqs_build_pauli without the device upload: the handle serves
 * nnqs_ham_info, nnqs_ham_export and nnqs_coupled_host only (calls that need
 * device tables return NNQS_E_INVAL).  Needs no GPU. */
nnqs_status nnqs_build_pauli_host(int n_spatial, const double *h, const double *eri, double e_core,
                                  double drop_tol, nnqs_ham **out);

/* info[0..5] (host) = n_qubits, n_words W, n_terms N_h, n_groups N_XY,
 * largest group size, device bytes held by the handle. */
nnqs_status nnqs_ham_info(const nnqs_ham *H, int64_t info[6]);

/* Host copies of the grouped tables (Alg. 1 output): xy[N_XY][W] group X/Y
 * masks, off[N_XY+1] CSR term offsets, yz[N_h][W] term Y/Z masks, coef[N_h]
 * folded coefficients.  Any pointer may be NULL to skip that table. */
nnqs_status nnqs_ham_export(const nnqs_ham *H, uint64_t *xy, int64_t *off, uint64_t *yz,
                            double *coef);

void nnqs_ham_free(nnqs_ham *H);

/* Ungrouped copy of the Hamiltonian for the layout comparison of Sec. 3.4:
 * the X/Y mask of every string ([n_terms][W] uint64, device memory owned by
 * the handle, freed by nnqs_ham_free).  Synchronous; idempotent.  Errors:
 * NNQS_E_INVAL (null handle or no device tables), NNQS_E_CUDA. */
nnqs_status nnqs_ham_build_ungrouped(nnqs_ham *H);

/* Bytes of the two layouts of the same strings (Sec. 3.4, Alg. 1):
 *   bytes[0] grouped, packed masks: per group W words + 4-byte offset +
 *            1-byte spin code, per string W words (Y/Z) + 8-byte coefficient;
 *   bytes[1] ungrouped, packed: per string 2W words (X/Y, Y/Z) + 8 bytes;
 *   bytes[2] grouped with one byte per qubit: per group N + 4, per string
 *            N + 8;
 *   bytes[3] ungrouped with one byte per qubit: per string 2N + 4 + 8.
 * Host only. */
nnqs_status nnqs_ham_layout_bytes(const nnqs_ham *H, int64_t bytes[4]);

/* ------------------------------------------------------------------ */
/* Ansatz: transformer amplitude + MLP phase (Sec. 3.1), number mask    */
/* (Sec. 3.3).                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n_qubits;     /* N, even, <= 128 */
    int32_t n_alpha;      /* electrons of each spin (mask of Sec. 3.3) */
    int32_t n_beta;
    int32_t d_model;      /* embedding width d, multiple of n_heads */
    int32_t n_layers;     /* decoder layers */
    int32_t n_heads;
    int32_t phase_hidden; /* phase MLP width (N x H x H x 1) */
    int32_t reserved;     /* must be 0 */
} nnqs_model_cfg;

typedef struct nnqs_model nnqs_model;

/* Parameters live in ONE caller-owned FP32 device array in this order
 * (Linear weights [out][in], row-major):
 *   tok_emb[5][d] pos_emb[T][d]                       (T = N/2)
 *   per layer l: ln1.g[d] ln1.b[d] attn.wqkv[3d][d] attn.bqkv[3d]
 *                attn.wo[d][d] attn.bo[d] ln2.g[d] ln2.b[d]
 *                ffn.w1[4d][d] ffn.b1[4d] ffn.w2[d][4d] ffn.b2[d]
 *   lnf.g[d] lnf.b[d] head.w[4][d] head.b[4]
 *   phase.w1[H][N] phase.b1[H] phase.w2[H][H] phase.b2[H] phase.w3[1][H] phase.b3[1]
 * The network: token t holds spatial orbital n-1-t as 2*y_beta + y_alpha;
 * the input sequence is a start token (id 4) then tokens 0..T-2; pre-LN
 * decoder layers with causal multi-head attention and a 4d erf-GELU FFN;
 * final LayerNorm (eps 1e-5); a d->4 head; the Sec. 3.3 mask (caps and
 * reachability) and a renormalised softmax give pi~(x_t | x_<t);
 * log|psi| = 1/2 sum_t log pi~; phase = MLP(x) with ReLU on the 0/1
 * occupations in qubit order. */
nnqs_status nnqs_model_create(const nnqs_model_cfg *cfg, nnqs_model **out);
void nnqs_model_free(nnqs_model *M);
int64_t nnqs_model_param_count(const nnqs_model *M);
/* offset/numel (host) of the named tensor, names as listed above */
nnqs_status nnqs_model_param_offset(const nnqs_model *M, const char *name, int64_t *offset,
                                    int64_t *numel);

size_t nnqs_logpsi_workspace_size(const nnqs_model *M, int64_t n, int prec);

/* (log|psi|, phase) of n packed bitstrings x (device, [n][W]) into out
 * (device, [n][2] double).  A bitstring outside the sector gets
 * log|psi| = -inf and sets NNQS_E_SECTOR in the workspace status. */
nnqs_status nnqs_logpsi(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n,
                        int prec, double *out, void *workspace, size_t workspace_bytes,
                        nnqs_stream stream);

size_t nnqs_logpsi_backward_workspace_size(const nnqs_model *M, int64_t n, int prec);

/* Reverse mode of nnqs_logpsi:
 *   grad = sum_i seed[i][0] d log|psi_i| / d theta + seed[i][1] d phase_i / d theta
 * seed device [n][2] double.  The gradient is written (overwritten) to
 * grad_f64 (device, double [P]) and/or grad_f32 (device, float [P]); at
 * least one must be non-NULL.  Accumulation is in FP64 for NNQS_FP64 and
 * FP32 otherwise.  Recomputes the forward (no activations are kept between
 * calls); samples are processed in chunks whose activations fit the
 * workspace. */
nnqs_status nnqs_logpsi_backward(const nnqs_model *M, const float *params, const uint64_t *x,
                                 int64_t n, int prec, const double *seed, double *grad_f64,
                                 float *grad_f32, void *workspace, size_t workspace_bytes,
                                 nnqs_stream stream);

/* ------------------------------------------------------------------ */
/* Local energy, Eq. (Eloc), with Alg. 2's fused evaluation (Sec. 3.4).  */
/* ------------------------------------------------------------------ */
size_t nnqs_eloc_workspace_size(const nnqs_ham *H, const nnqs_model *M, int64_t n_lut,
                                int64_t n_rows, int mode, int prec);

/* E_loc(x) = sum_{x'} H_{x x'} psi(x')/psi(x) for x = lut[row_begin + i],
 * i < n_rows, written to eloc_out (device, [n_rows][2] double).
 *   lut         device [n_lut][W]: the unique samples S (any order, no
 *               duplicates, all in the (n_alpha, n_beta) sector)
 *   lut_logpsi  device [n_lut][2]: (log|psi|, phase) of each lut row; read
 *               in NNQS_SA mode, ignored in NNQS_EXACT mode
 *   M, params   the ansatz; required in NNQS_EXACT mode (log psi of every
 *               coupled x' and of x is computed with precision `prec`),
 *               ignored in NNQS_SA mode (may be NULL)
 *   flags       NNQS_SWEEP_* (NNQS_SA only)
 * NNQS_EXACT synchronises once to size the forward over the unique coupled
 * set; NNQS_SA is fully asynchronous. */
nnqs_status nnqs_eloc(const nnqs_ham *H, const nnqs_model *M, const float *params,
                      const uint64_t *lut, const double *lut_logpsi, int64_t n_lut,
                      int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int mode,
                      int prec, int flags, double *eloc_out, void *workspace,
                      size_t workspace_bytes, nnqs_stream stream);

/* nnqs_eloc in NNQS_SA mode for callers that cannot allocate device memory:
 * code running inside a host application that owns the GPU's memory (a
 * framework whose pool has reserved the device, a plugin interface that
 * hands out no allocator) cannot provide a workspace, and cudaMalloc itself
 * synchronises the device, which a latency-bound caller cannot afford.  This
 * entry point takes no workspace and allocates nothing: its scratch is one
 * fixed 64 MiB array in device memory that every GPU loading the library
 * holds until the process exits.  The paper has no counterpart: this is a
 * calling convention, not part of the method.
 *   Arguments, argument checks and result as nnqs_eloc (mode NNQS_SA),
 *   every NNQS_SWEEP_* flag included (NNQS_SWEEP_TERMS after
 *   nnqs_ham_build_ungrouped).  The scratch a call needs is sized for the
 *   sweep that call runs (NNQS_SWEEP_AUTO resolved first): 65 to 145 bytes
 *   per table row, depending on the table size (the hash has a power-of-two
 *   capacity) and the word count, so tables of about 5 x 10^5 rows fit; a
 *   call above 64 MiB is rejected
 *   with NNQS_E_INVAL before any launch; use nnqs_eloc with a workspace then.
 *   check != 0: synchronise `stream` and return the status the kernels
 *   recorded (sample outside the sector, duplicate, ...).  check == 0: fully
 *   asynchronous, and errors the GPU detects are lost: the status word lives
 *   in the shared array only until the next call clears it, and there is no
 *   call to read it.  Callers that need those errors pass check != 0.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process; make that first call before any stream capture, and
 * do not reset the device's primary context (cudaDeviceReset) after it: the
 * kept address would then be stale.  All calls share the one array, which
 * keeps the previous call's contents (each call clears what must start at
 * zero): calls whose execution overlaps on the GPU -- from two streams, or
 * two host threads -- race on it and must be serialised by the caller. */
nnqs_status nnqs_eloc_sa_noalloc(const nnqs_ham *H, const uint64_t *lut, const double *lut_logpsi,
                                 int64_t n_lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                                 int n_beta, int flags, double *eloc_out, int check,
                                 nnqs_stream stream);

/* The coupled set of exact mode exactly as the GPU builds it for nnqs_eloc
 * (mode NNQS_EXACT), exported for parity tests and inspection (Eq. Eloc over
 * every x' with H_{x x'} != 0 structurally; the dedup of Sec. 3.4 (2)): the
 * rows x = lut[row_begin + i], i < n_rows, and every x' = x ^ m over the
 * groups m that keep the (n_alpha, n_beta) sector are inserted into the
 * device hash table and numbered, as nnqs_eloc does before its forward.
 * Outputs (device, caller-owned):
 *   unique_out  [cap_unique][W]: the distinct keys U (rows and their coupled
 *               states, each once) in the table's slot order (unspecified);
 *               *n_unique_out (host) receives |U|
 *   row_count   [n_rows] int32: number of coupled x' of row i (the identity
 *               group included, so x itself is one of them)
 *   row_idx     [n_rows][row_cap] int32: index into U of each coupled x' of
 *               row i, in group order (ascending X/Y mask)
 *   row_hxx     [n_rows][row_cap] double: H_{x x'} of those x'
 * Errors: NNQS_E_INVAL (arguments; cap_unique < |U|, *n_unique_out still
 * set), NNQS_E_WORKSPACE; device-detected (nnqs_workspace_status): a row
 * outside the sector (NNQS_E_SECTOR), a row with more than row_cap coupled
 * states (NNQS_E_TABLE_FULL; its count is still written).  Synchronises once
 * (to read |U|).  Workspace: nnqs_exact_coupled_workspace_size. */
size_t nnqs_exact_coupled_workspace_size(const nnqs_ham *H, int64_t n_rows);
nnqs_status nnqs_exact_coupled(const nnqs_ham *H, const uint64_t *lut, int64_t n_lut, int64_t row_begin,
                               int64_t n_rows, int n_alpha, int n_beta, uint64_t *unique_out,
                               int64_t cap_unique, int64_t *n_unique_out, int32_t *row_count,
                               int32_t *row_idx, double *row_hxx, int64_t row_cap, void *workspace,
                               size_t workspace_bytes, nnqs_stream stream);

/* Coupled set of one row (parity and debugging): every x' = x ^ m over the
 * groups m that keep the sector, in group order, with H_{x x'} (host
 * outputs, at most `cap` entries; *count receives the number).  Host-side,
 * synchronous. */
nnqs_status nnqs_coupled_host(const nnqs_ham *H, const uint64_t *x, int n_alpha, int n_beta,
                              uint64_t *xp, double *hxx, int64_t cap, int64_t *count);

/* ------------------------------------------------------------------ */
/* Energy, variance and gradient (Sec. 2.1, Eqs. energy and the          */
/* gradient estimator).                                                  */
/* ------------------------------------------------------------------ */
size_t nnqs_energy_stats_workspace_size(int64_t n);

/* stats (device, 4 doubles) = Re E, Im E, Var, sum w with
 * E = sum_i w_i E_loc,i / sum_i w_i and Var = sum_i w_i |E_loc,i - E|^2 / sum w.
 * eloc device [n][2]; weights device [n] uint64 sample counts. */
nnqs_status nnqs_energy_stats(const double *eloc, const uint64_t *weights, int64_t n,
                              double *stats, void *workspace, size_t workspace_bytes,
                              nnqs_stream stream);

size_t nnqs_energy_grad_workspace_size(const nnqs_ham *H, const nnqs_model *M, int64_t n_u,
                                       int prec);

/* One energy/gradient evaluation on the unique samples S with counts w:
 * log psi(S) -> sample-aware E_loc (Alg. 2) -> stats -> gradient
 * grad = 2 Re sum_i w_i (E_loc,i - E) d ln psi_i^* / sum w  (Sec. 2.1, with
 * E_loc held fixed and E the complex weighted mean).  Outputs (device):
 * stats[4] as nnqs_energy_stats, eloc_out [n_u][2] (may be NULL),
 * grad_f64 / grad_f32 as nnqs_logpsi_backward (at least one non-NULL). */
nnqs_status nnqs_energy_grad(const nnqs_ham *H, const nnqs_model *M, const float *params,
                             const uint64_t *samples, const uint64_t *weights, int64_t n_u,
                             int prec, double *stats, double *eloc_out, double *grad_f64,
                             float *grad_f32, void *workspace, size_t workspace_bytes,
                             nnqs_stream stream);

/* ------------------------------------------------------------------ */
/* Batch autoregressive sampling (Sec. 3.1 BAS, mask of Sec. 3.3).       */
/* ------------------------------------------------------------------ */
/* nnqs_sample flags: by default each step evaluates only the new token of
 * every prefix against a key/value cache of the prefix tree (each node keeps
 * its own rows; memory T * max_unique * n_layers * 3 d values);
 * NNQS_SAMPLE_RECOMPUTE re-runs the whole prefix at every step instead (no
 * cache).  Both give bit-identical draws.
 * NNQS_SAMPLE_KEEP (with the cache; BF16 or split-BF16 arithmetic, d_model
 * 64, max_unique <= 65536, else NNQS_E_UNSUPPORTED) also keeps in the
 * workspace, for every tree node the decode visits, its residual row at each
 * layer's input and after each layer's attention and its final residual
 * (2 L + 1 rows of d_model floats per node, T max_unique + 1 nodes), and the
 * last level's ancestor table: what nnqs_energy_grad_sampled reads instead of
 * running the forward again.  The draws are the same with or without it. */
enum { NNQS_SAMPLE_RECOMPUTE = 1, NNQS_SAMPLE_KEEP = 2 };

size_t nnqs_sample_workspace_size(const nnqs_model *M, int64_t max_unique, int prec, int flags);

/* Draws n_samples samples from |psi|^2 as unique bitstrings with counts:
 * at each of the T steps every unique prefix with weight w splits w over
 * its 4 children by a multinomial draw from pi~ (sequential binomials on a
 * Philox4x32-10 counter stream keyed by (seed, step, prefix)); zero-weight
 * children are pruned.  Outputs (device) samples_out [max_unique][W] and
 * weights_out [max_unique]; *n_unique_out (host) = unique samples written,
 * sorted ascending.  Returns NNQS_E_TABLE_FULL if a step holds more than
 * max_unique prefixes.  With the key/value cache, BF16 or split-BF16
 * arithmetic, d_model = 64, max_unique <= 65536 and one activation chunk,
 * the level sizes stay on the device and the stream is synchronised once at
 * the end (to return *n_unique_out); otherwise once per step (the width of
 * the next step is data-dependent). */
nnqs_status nnqs_sample(const nnqs_model *M, const float *params, uint64_t n_samples,
                        uint64_t seed, int prec, int flags, int64_t max_unique,
                        uint64_t *samples_out, uint64_t *weights_out, int64_t *n_unique_out,
                        void *workspace, size_t workspace_bytes, nnqs_stream stream);

/* nnqs_energy_grad with the forward's quantities taken from the tree the
 * last nnqs_sample call with NNQS_SAMPLE_KEEP left in sample_workspace
 * (sample_workspace_bytes, max_unique and prec as in that call), instead of
 * running the forward again: each token row's layer inputs and mid residuals
 * are its tree node's, the final LayerNorm, head and log|psi| follow from
 * them, the phase MLP and the local energy run as in nnqs_energy_grad, and
 * the reverse mode is the fused one (Sec. 2.1 gradient estimator).
 * samples / weights / n_u: that call's outputs, unmodified and in its order
 * (a row that differs records NNQS_E_INVAL in the workspace status).  Same
 * outputs, layout and errors as nnqs_energy_grad; NNQS_E_UNSUPPORTED outside
 * BF16 / split-BF16 arithmetic, d_model 64, FFN width 256, head dimension 8
 * or 16, T <= 64 (the fused reverse mode's reach); NNQS_E_WORKSPACE when
 * sample_workspace is smaller than an NNQS_SAMPLE_KEEP call needs.  The
 * sampler's workspace is only read. */
size_t nnqs_energy_grad_sampled_workspace_size(const nnqs_ham *H, const nnqs_model *M, int64_t n_u, int prec);
/* 1 if nnqs_sample with NNQS_SAMPLE_KEEP and nnqs_energy_grad_sampled apply
 * to this model, precision and max_unique, else 0 (host only). */
int nnqs_energy_grad_sampled_supported(const nnqs_model *M, int prec, int64_t max_unique);
nnqs_status nnqs_energy_grad_sampled(const nnqs_ham *H, const nnqs_model *M, const float *params,
                                     const void *sample_workspace, size_t sample_workspace_bytes,
                                     int64_t max_unique, const uint64_t *samples, const uint64_t *weights,
                                     int64_t n_u, int prec, double *stats, double *eloc_out, double *grad_f64,
                                     float *grad_f32, void *workspace, size_t workspace_bytes,
                                     nnqs_stream stream);

/* ------------------------------------------------------------------ */
/* Optimiser step.                                                       */
/* ------------------------------------------------------------------ */
/* Adam (no weight decay), in place on device FP32 arrays of length n;
 * `step` is the 1-based count after this update. */
nnqs_status nnqs_adam_step(float *params, const float *grad, float *m, float *v, int64_t n,
                           int64_t step, double lr, double beta1, double beta2, double eps,
                           nnqs_stream stream);

/* AdamW (Sec. 4.1 trains with it): Adam with decoupled weight decay,
 * theta <- theta * (1 - lr * weight_decay), then the Adam step of
 * nnqs_adam_step with the same arguments.  Same layout, ownership and
 * errors as nnqs_adam_step; NNQS_E_INVAL also when weight_decay < 0 or
 * lr * weight_decay >= 1.  weight_decay = 0 gives nnqs_adam_step. */
nnqs_status nnqs_adamw_step(float *params, const float *grad, float *m, float *v, int64_t n,
                            int64_t step, double lr, double beta1, double beta2, double eps,
                            double weight_decay, nnqs_stream stream);

/* Learning rate of training step `step` (1-based) under the warm-up schedule
 * of Sec. 4.1: d_model^-0.5 * min(step^-0.5, step * warmup^-1.5); it rises
 * linearly to its peak (d_model * warmup)^-0.5 at step = warmup and decays as
 * step^-0.5 after.  Host only, no device work; 0 for step < 1, d_model < 1 or
 * warmup < 1. */
double nnqs_lr_warmup(int64_t step, int d_model, int64_t warmup);

#ifdef __cplusplus
}
#endif
#endif /* NNQS_H */
