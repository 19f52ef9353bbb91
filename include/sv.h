/*
 * sv.h -- C interface of the GB300 (sm_103a) state-vector simulator of random lattice
 * ("supremacy") circuits, after Li, Wu, Ying, Sun, Yang, "Quantum Supremacy Circuit
 * Simulation on Sunway TaihuLight" (arXiv:1804.04797).
 *
 * Conventions (all calls)
 *   - Amplitude order: |psi> = (alpha_0 .. alpha_{2^n-1}) and qubit k is bit k of the
 *     index (§2, the pair-update equation).  The state lives on the device as 2^n
 *     interleaved complex64 values {float re, float im}.
 *   - Bitstrings are uint64_t, bit q = outcome of qubit q.
 *   - Every call returns sv_status; on failure sv_last_error() (thread-local) gives a
 *     one-line message.  No call keeps a host pointer after it returns.  The library
 *     owns the device memory it allocates; the caller owns every host array.
 *   - Calls are ordered on the handle's CUDA stream.  Calls that return host data
 *     (amplitudes, norms, branch amplitudes, batch statistics) synchronise it.
 *   - There is no CPU fallback: without a usable CUDA device, calls that touch the
 *     device return SV_ERR_CUDA.  sv_generate_circuit and sv_plan_* are host-only.
 */
#ifndef PAPER_1804_04797_GB300_SV_H_
#define PAPER_1804_04797_GB300_SV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SV_OK = 0,
  SV_ERR_ARG = 1,     /* invalid argument: size, qubit index, gate kind, pointer      */
  SV_ERR_OOM = 2,     /* a device allocation failed; the state is left unchanged      */
  SV_ERR_CUDA = 3,    /* a CUDA call failed (message holds cudaGetErrorString)        */
  SV_ERR_TIMEOUT = 4, /* a bounded in-kernel wait gave up (no hang; device flag read)  */
  SV_ERR_STATE = 5    /* the handle is unusable after an earlier failed apply          */
} sv_status;

/* Gate kinds.  H, T, SX = X^{1/2}, SY = Y^{1/2} and CZ are the gate set of §2 (the
 * paragraph after Fig. 2).  Matrices (the paper prints none; the principal roots):
 *   H  = [[1,1],[1,-1]]/sqrt2          T  = diag(1, e^{i pi/4})
 *   SX = [[1+i,1-i],[1-i,1+i]]/2       SY = [[1+i,-1-i],[1+i,1+i]]/2
 *   CZ = diag(1,1,1,-1) on (q0, q1)
 * P0 = |0><0|, P1 = |1><1| (the projectors of §2.1) and Z = diag(1,-1) are the product
 * terms of the decomposition CZ = P0 (x) I + P1 (x) Z (§2, Fig. 2).  TDG, SXDG, SYDG are
 * the adjoints of T, SX, SY (for inverse circuits). */
typedef enum {
  SV_H = 0, SV_T = 1, SV_SX = 2, SV_SY = 3, SV_CZ = 4,
  SV_P0 = 5, SV_P1 = 6, SV_Z = 7, SV_TDG = 8, SV_SXDG = 9, SV_SYDG = 10
} sv_kind;

/* One gate; q1 is read for CZ only.  layer is informational (0 = the H layer). */
typedef struct {
  uint8_t kind, q0, q1, pad;
  uint32_t layer;
} sv_gate;

/* Arithmetic of the in-tile update. */
enum {
  SV_PREC_PLAIN = 0,  /* fp32 CUDA-core arithmetic, one gate at a time (the square    */
                      /* roots as rotations, their scalar applied once per plan)      */
  SV_PREC_TF32X3 = 1, /* fused k-qubit unitaries on tcgen05 tensor cores, 3-pass     */
                      /* split-TF32 products (hi*hi + hi*lo + lo*hi), fp32 accumulate */
  SV_PREC_F16X3 = 2,  /* the same with fp16 hi/lo parts (same 11-bit significand,     */
                      /* twice the tensor rate; rows scaled by powers of two)          */
                      /* Both tensor-core modes need tiles of 12 or 13 qubits: a      */
                      /* state below 12 qubits runs the plain kernel instead, and     */
                      /* sv_profile.plain_fallbacks counts those applies.             */
  SV_PREC_PERGATE = 3 /* one full sweep of the state per gate (no tiling; baseline)  */
};

/* Options.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  int fuse_k;     /* qubits per register group besides qubit 0 (plain) or per fused   */
                  /* block (tensor cores), 1..5; 0 = the default 5 (plain kernels     */
                  /* compiled per plan use at most 4).  The tensor-core precisions    */
                  /* take 5 (32x32 stage unitaries) or 4 (16x16, 12-qubit tiles only);  */
                  /* any other value is SV_ERR_ARG.                                    */
  int precision;  /* SV_PREC_*                                            [PLAIN]       */
  int autotune;   /* 1 = pick shapes by timing, kept in a JSON cache (SV_AUTOTUNE_CACHE, */
                  /* default autotune.json beside the library) [0].  sv_apply_circuit  */
                  /* on a fresh state with plan-specialised kernels and tile_bits 0:   */
                  /* the tile size and the fusion width -- 12- or 13-qubit tiles with  */
                  /* 5-qubit stages, or 12-qubit tiles with 6-qubit stages (fuse_k 0   */
                  /* only; otherwise the width stays fuse_k) -- and each pass's        */
                  /* compute groups of the pipelined kernel, timed on the circuit      */
                  /* itself (its first call runs the candidate plans a few times);     */
                  /* sv_apply_batch: the tile size.                                    */
  void *stream;   /* cudaStream_t used by the handle                      [legacy 0]    */
  int tile_bits;  /* qubits per gathered tile, 6..14 (14: plan-specialised kernels    */
                  /* only) [12 on plan-specialised and tensor-core kernels, 13 on the  */
                  /* interpreting kernel]                                              */
  int low_bits;   /* contiguous low qubits in every tile (coalescing)     [4]           */
  int jit;        /* plain path: run each plan on kernels compiled for it at run time */
                  /* (NVRTC; cached in memory and in the library's directory):       */
                  /* 1 = always (error if NVRTC fails), -1 = never, 0 = for n >= 24 [0] */
                  /* (sv_apply_batch: per circuit, see there)                         */
  int pipeline;   /* plain path on plan-specialised kernels: 0 = the pipelined         */
                  /* persistent kernel (one CTA per SM; a producer warp streams tiles  */
                  /* into a ring of shared-memory slots with TMA tensor copies while   */
                  /* compute groups run the stages) wherever the tile shape allows it  */
                  /* (10..13 tile qubits, low_bits 4) [0]; -1 = one CTA per tile in    */
                  /* flight, tile read with per-thread asynchronous copies             */
  int norm_restore; /* tensor-core precisions: 0 = restore every tile's norm in the    */
                  /* pass's last stage (unbiased stochastic rounding; the tensor      */
                  /* cores' fp32 accumulation truncates toward zero, ~1e-7 per stage)  */
                  /* [0]; -1 = leave the products as the tensor cores computed them    */
                  /* (the raw error; the norm is then a check, not a correction)       */
} sv_options;

/* An R x C lattice circuit: bit r*cols+c of removed_mask drops site (r,c); kept sites
 * are numbered row-major.  depth counts layers after the layer-0 H gates (§1 footnote). */
typedef struct {
  int rows, cols;
  uint64_t removed_mask;
  int depth;
  uint64_t seed;
} sv_lattice;

/* A cut of the qubits into halves A (bits set) and B.  full_decomposition = 1 expands
 * every crossing CZ into both product terms (no implicit decomposition, no phase
 * absorption; the plain reading of Eq. 1). */
typedef struct {
  uint64_t half_a_mask;
  int full_decomposition;
  int depth;  /* sv_branch_full_state: 0 = every layer in the two halves; d > 0 = layers     */
              /* 0..d in the halves (parts A and B of §2.1, Fig. 2), the layers after d   */
              /* (part C, Eq. 3) applied to the reconstructed full state.  Must be 0 for  */
              /* sv_branch_amplitudes and sv_branch_counts.                               */
} sv_cut;

typedef struct sv_state sv_state;

/* Thread-local text of the last error ("" if none).  Valid until the next call. */
const char *sv_last_error(void);

/* --- state lifetime -------------------------------------------------------------- */

/* Allocate a 2^n complex64 state in |0...0> (§2 initial state).  1 <= n <= 34 (34
 * qubits = 128 GiB).  opts may be NULL.  Returns SV_ERR_OOM if cudaMalloc fails. */
sv_status sv_create(int n_qubits, const sv_options *opts, sv_state **out);

/* Wrap a caller-owned device buffer of 2^n complex64 (e.g. a torch tensor).  The
 * buffer must stay alive until sv_destroy, which does not free it.  Its content is
 * taken as the current state.  stream may be NULL (legacy default stream). */
sv_status sv_create_from_ptr(int n_qubits, void *dev_ptr, void *stream, sv_state **out);

/* Release the handle and the device memory it owns.  NULL is accepted. */
sv_status sv_destroy(sv_state *s);

/* Replace the options (precision, fusion width, tile shape, stream). */
sv_status sv_set_options(sv_state *s, const sv_options *opts);

/* Copy the 2^n complex64 amplitudes to dst (host or device memory, 8*2^n bytes). */
sv_status sv_copy_state(sv_state *s, void *dst);

/* Overwrite the state with 2^n complex64 values from src (host or device memory). */
sv_status sv_load_state(sv_state *s, const void *src);

/* Return the state to |0...0> without touching the device: the next apply generates
 * the initial state in its first pass instead of reading the buffer. */
sv_status sv_reset(sv_state *s);

/* Device pointer of the amplitudes (owned by the handle or the caller).  The caller
 * may read or write the amplitudes through it between calls on the handle's stream; from
 * then on sv_norm always reduces the state itself (sums formed by earlier passes are not
 * reused). */
sv_status sv_device_ptr(sv_state *s, void **ptr);

/* --- circuits ---------------------------------------------------------------------- */

/* Seeded lattice circuit (§2: gates H, T, X^{1/2}, Y^{1/2}, CZ on lattice neighbours,
 * fixed CZ positions per layer; layer-0 H on every qubit).  Rules: 8 CZ patterns used
 * cyclically (horizontal bond (r,c)-(r,c+1) in class (c+2(r mod 2)) mod 4, vertical bond
 * (r,c)-(r+1,c) in class (r+2(c mod 2)) mod 4, layer l uses [H0,V0,H1,V1,H2,V2,H3,V3][(l-1)
 * mod 8]); in layer l a qubit that was in a CZ of layer l-1 and is in none of layer l
 * gets one of {T, SX, SY} different from its previous one, drawn by SplitMix64(seed)
 * (layers, then qubits ascending; candidates [T,SX,SY] minus the previous one; pick
 * draw % count).  Within a layer: one-qubit gates by qubit, then CZs by (q0<q1).
 * Writes at most cap gates to out (out may be NULL to query *n_out).  Host only.
 * SV_ERR_ARG if the lattice has more than 64 sites, or cap is too small. */
sv_status sv_generate_circuit(const sv_lattice *lat, sv_gate *out, size_t cap, size_t *n_out);

/* Apply gates in list order (§2 pair update for one-qubit gates, diagonal CZ).  The
 * list is planned into passes over 2^tile_bits-amplitude gathered tiles and k-qubit
 * groups (the bunching of gates on "local qubits" of §2.3, generalised to any qubit
 * set).  If the state is still the initial |0..0> and the list starts with H on every
 * qubit, that layer becomes the uniform amplitude 2^{-n/2} written by the first pass.
 * The same list, options and starting condition as the handle's previous call reuse that
 * call's plan and kernels.  On plan-specialised kernels (sv_options.jit) the last pass
 * also forms the fp64 norm sums that sv_norm then returns.
 * SV_ERR_ARG for a qubit >= n, CZ with q0 == q1, or an unknown kind (state untouched).
 * A CUDA failure marks the handle SV_ERR_STATE. */
sv_status sv_apply_circuit(sv_state *s, const sv_gate *gates, size_t n_gates);

/* Apply the inverse of the gate list (reverse order, adjoint of each gate). */
sv_status sv_apply_circuit_inverse(sv_state *s, const sv_gate *gates, size_t n_gates);

/* alpha_x for m bitstrings, written as 2m doubles (re, im).  Bits >= n must be 0. */
sv_status sv_get_amplitudes(sv_state *s, const uint64_t *bits, size_t m, double *out_re_im);

/* fp64 sums over the state: norm2 = sum |alpha|^2, sum_p2 = sum |alpha|^4 (the
 * Porter-Thomas statistic of §3: N * sum_p2 -> 2).  Either pointer may be NULL.
 * Deterministic (fixed two-level tree).  After sv_apply_circuit on plan-specialised
 * kernels (sv_options.jit) the sums were formed by the pass that wrote the state and the
 * call reads no state; any other write of the state (reset, load, basis state, a
 * sv_device_ptr or sv_create_from_ptr state) makes it reduce the state again. */
sv_status sv_norm(sv_state *s, double *norm2, double *sum_p2);

/* Allocation-free variant of sv_norm, for callers that cannot allocate device memory:
 * code under a device-memory budget owned by another allocator (a framework's caching
 * allocator that has reserved the GPU), or code that must avoid the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this is a
 * library-usage convenience.
 *   dev_state  2^n_qubits complex64 amplitudes on the current device (caller-owned),
 *              16-byte aligned (8-byte for n_qubits = 1): the reduction reads two
 *              amplitudes per vector load; a misaligned pointer is SV_ERR_ARG.
 *   n_qubits   1..34; anything else is SV_ERR_ARG.
 *   stream     cudaStream_t to run on (NULL = legacy default stream); synchronised.
 *   norm2, sum_p2  host doubles for sum |alpha|^2 and sum |alpha|^4 (either may be NULL).
 * The scratch is one fixed file-scope device array of 1024 partial sums (16 KB + 16 B)
 * that every GPU loading the library keeps until the process exits; the call makes no
 * cudaMalloc/cudaFree.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current: make it before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls that overlap
 * on the GPU (other streams or host threads) race and can return wrong sums. */
sv_status sv_norm_noalloc(const void *dev_state, int n_qubits, void *stream, double *norm2, double *sum_p2);

/* Probabilities |alpha_x|^2 for m indices, in fp64. */
sv_status sv_get_probabilities(sv_state *s, const uint64_t *bits, size_t m, double *out);

/* --- few-amplitude task -------------------------------------------------------------- */

/* alpha_x for m bitstrings of the lattice circuit by the cut decomposition (§2, Fig. 2
 * and Eq. 1): every CZ with one qubit in each half is replaced by its two product terms
 * (P_l on one qubit, Z^l on the other); all branches of a half run as one batched state
 * (branch bits are extra index bits), and alpha_x = sum_l A_l[x_A] * B_l[x_B] is summed
 * in fp64.  Unless cut->full_decomposition: a crossing CZ after which neither qubit meets
 * a non-diagonal gate is a sign (-1)^{x_a x_b} of the output (§3: the last layer's CZs
 * only change phases) and is not expanded; one after which only one qubit stays in its
 * basis state gets the projector on that qubit, and that half needs no branch bit for it
 * (§2.1 implicit decomposition: its branch index is the qubit's output bit).  Halves plus
 * their branch bits of at most 34 qubits.  out_re_im: 2m doubles.  opts may be NULL. */
sv_status sv_branch_amplitudes(const sv_lattice *lat, const sv_cut *cut, const uint64_t *bits,
                               size_t m, const sv_options *opts, double *out_re_im);

/* The full state from the cut decomposition in tensor form (§2, Eqs. 6-7), continued by
 * the circuit's part C when cut->depth > 0 (Eq. 3: the decomposed layers 0..depth give the
 * state psi_AB, the remaining layers run on it as ordinary passes): the two
 * halves' batched branch states A (n_A + t qubits) and B (n_B + t) give
 * psi[x_A + (x_B << n_A)] = sum_l A_l[x_A] B_l[x_B], a complex matrix product over the
 * 2^t branches, written into out (an n-qubit handle on the same device; fp32
 * accumulation).  Crossing CZs that only sign the output are applied to the result as
 * CZ gates; the others are fully decomposed (an implicit decomposition fixes a branch by
 * an output bit, which a product over all outputs cannot).  Half A must be qubits
 * 0..n_A-1 (a cut between lattice rows).  SV_ERR_ARG otherwise. */
sv_status sv_branch_full_state(const sv_lattice *lat, const sv_cut *cut, const sv_options *opts, sv_state *out);

/* The decomposition sv_branch_amplitudes runs for a cut (host only): counts[0] = CZs
 * crossing the cut, [1] = those absorbed as output signs, [2] = branch bits of half A,
 * [3] = of half B, [4] = branch bits summed over (2^counts[4] terms per amplitude). */
sv_status sv_branch_counts(const sv_lattice *lat, const sv_cut *cut, int counts[5]);

/* --- batch ------------------------------------------------------------------------------ */

/* Simulate count independent lattice circuits (each with its own state, 6..28 qubits;
 * §2's circuits at many sizes) in ONE persistent launch over a work queue of (circuit,
 * pass, tile) items: all circuits' first passes, then all second passes, ...  An item
 * waits for its circuit's previous pass with a bounded spin; if a wait gives up the call
 * returns SV_ERR_TIMEOUT (no hang).  The launch, the queue reset and the per-circuit fp64
 * statistics are captured once in a CUDA graph and replayed while the same lattice list
 * is passed again; the states stay on the device until the next different batch or
 * sv_batch_free.  opts (may be NULL): tile_bits 0 or 10..13 (default 13); autotune = 1
 * with tile_bits 0 times tile sizes 11..13 on this batch and keeps the fastest in a JSON
 * cache (SV_AUTOTUNE_CACHE, default autotune.json beside the library); stream orders the
 * call after the caller's stream; jit 0 runs the circuits of 24 or more qubits (jit 1:
 * of 12 or more; -1: none) on kernels compiled for their plans, each pass its own launch
 * recorded in the same graph after the persistent one (with jit 0 and no NVRTC they join
 * the persistent launch).  stats_out: 3 doubles per circuit, [sum |alpha|^2,
 * sum |alpha|^4, n_qubits]; NULL skips the statistics (a second graph, without the
 * reduction over all states, is captured for such calls).  Synchronises. */
sv_status sv_apply_batch(const sv_lattice *circs, size_t count, const sv_options *opts,
                         double *stats_out);

/* Amplitudes of circuit `circuit` of the last batch (host doubles re, im; 2m values). */
sv_status sv_batch_amplitudes(size_t circuit, const uint64_t *bits, size_t m, double *out_re_im);

/* Release the device memory and graph kept for the last batch. */
sv_status sv_batch_free(void);

/* The configuration the last batch ran with (host ints, any may be NULL): tile_bits =
 * the tile size of its persistent launch (the autotuner's choice when it was asked for),
 * plan_kernel_circuits = the circuits run on plan-specialised kernels, persistent_circuits
 * = the circuits in the persistent launch.  SV_ERR_STATE if no batch has run. */
sv_status sv_batch_config(int *tile_bits, int *plan_kernel_circuits, int *persistent_circuits);

/* Failure-detection self-test, with no GPU fault: runs the batch kernel on a queue whose
 * single item waits for a pass that is never queued, with a wait limit of limit_ms
 * (1..10000).  Returns SV_ERR_TIMEOUT when the kernel gave up and reported it as designed
 * (the expected result); SV_OK would mean the bounded wait did not fire. */
sv_status sv_selftest_wait_timeout(int limit_ms);

/* --- planning and measurement (host-only helpers) --------------------------------------- */

typedef struct {
  int passes;         /* HBM sweeps of the state (including the write-only init, if any) */
  int stages;         /* k-qubit groups over all passes                                   */
  int ops;            /* gate operations after planning                                   */
  int init_uniform;   /* 1 if the layer-0 H gates became the uniform first pass           */
  double hbm_bytes;   /* algorithmic bytes of the passes: 16 * 2^n per read-write pass,   */
                      /* 8 * 2^n for the write-only first pass                             */
  int matrix_stages;  /* stages with gates inside their register qubits (on the tensor-    */
                      /* core path: one 32x32 complex product per tile each)               */
} sv_plan_summary;

/* Plan a gate list for an n-qubit state without touching the device.  order_out (may
 * be NULL, else n_gates entries) receives the gate indices in execution order;
 * pass_out (may be NULL) the pass of each executed gate; tile_out (may be NULL, else
 * 64 * passes entries) the qubits of each pass's tile (-1 padded). */
sv_status sv_plan(int n_qubits, const sv_gate *gates, size_t n_gates, const sv_options *opts,
                  int fresh_state, sv_plan_summary *summary, int32_t *order_out,
                  int32_t *pass_out, int32_t *tile_out, size_t tile_cap);

/* Per-kernel timing collected with CUDA events on the handle's stream while enabled. */
typedef struct {
  int launches;       /* tile-pass (or per-gate) kernel launches                 */
  double ms;          /* their summed device time                                */
  double hbm_bytes;   /* their summed algorithmic bytes                          */
  double h2d_bytes;   /* host-to-device bytes copied by the library (plans, indices) */
  double d2h_bytes;   /* device-to-host bytes copied by the library (results)     */
  int other_launches; /* other kernels (reductions, gathers, init)               */
  int jit_launches;   /* tile passes run on plan-specialised (run-time compiled) kernels */
  int plain_fallbacks; /* applies with a tensor-core precision that ran the plain kernel */
                       /* (states below 12 qubits)                                    */
  int plan_tile_bits;    /* the last tile-pass plan: qubits per tile (the autotuner's   */
  int plan_stage_qubits; /* choice when it ran) and per stage (the fusion width); 0    */
  int plan_passes;       /* when no plan ran; its passes                                */
} sv_profile;

/* The basis state |x> (1 at index x, 0 elsewhere).  SV_ERR_ARG if x has bits >= n. */
sv_status sv_set_basis_state(sv_state *s, uint64_t x);

/* <a|b> = sum_i conj(a_i) b_i of two states of the same size on the same device, into
 * out_re_im[0..1] (fp64 accumulation of fp32 products: 8 products per fp32 chunk, chunk
 * sums in fp64).  Waits for b's stream, runs on a's and synchronises it. */
sv_status sv_inner_product(sv_state *a, sv_state *b, double *out_re_im);

/* Task 2 by the inner product of two states (§2 "Calculating one or a few amplitudes",
 * the equation alpha_x = <phi|psi>): the lattice circuit U = U2 U1 is cut after layer
 * split_layer (U1 = layers 0..split_layer, the H layer included; U2 = the rest),
 * |psi> = U1 H^n |0> is computed once, and for every bitstring x, |phi_x> = U2^dagger |x>
 * and alpha_x = <phi_x|psi>; on plan-specialised kernels (sv_options.jit) the last pass
 * of phi_x sums <phi_x|psi> instead of storing phi_x.  Two n-qubit states are allocated
 * (2 x 8 x 2^n bytes, at most n = 34 on GB300) and freed on return; out_re_im receives
 * 2m doubles.  A split_layer at or beyond the depth gives the plain amplitudes of the
 * full state. */
sv_status sv_amplitudes_by_inner_product(const sv_lattice *lat, int split_layer, const uint64_t *bits, size_t m,
                                         const sv_options *opts, double *out_re_im);

/* Compile the plan-specialised kernels of a gate list for sm_103a without a device
 * (NVRTC only; no cache is read or written), and the last pass once more as the variant
 * that sums an inner product instead of storing (sv_amplitudes_by_inner_product): a check
 * of the code generator.  log (may
 * be NULL) receives up to log_cap bytes of the compiler's messages, NUL-terminated.
 * SV_ERR_CUDA when NVRTC is missing or the compile fails. */
sv_status sv_jit_check(int n_qubits, const sv_gate *gates, size_t n_gates, const sv_options *opts,
                       int fresh_state, char *log, size_t log_cap);

/* Turn the per-kernel timing of the handle on (on != 0, counters cleared) or off; it
 * records a CUDA event pair around every pass launch on the handle's stream. */
sv_status sv_set_profiling(sv_state *s, int on);
/* The counters since profiling was turned on (synchronises the handle's stream). */
sv_status sv_get_profile(sv_state *s, sv_profile *out);
/* Each timed launch since profiling was turned on, in launch order (synchronises the
 * handle's stream): *n_out = the number of launches; the first min(n, cap) entries of
 * ms_out (device time of the launch, CUDA events on the handle's stream) and bytes_out
 * (its algorithmic bytes) are written; either array may be NULL. */
sv_status sv_get_launch_times(sv_state *s, double *ms_out, double *bytes_out, size_t cap, size_t *n_out);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_1804_04797_GB300_SV_H_ */
