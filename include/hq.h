/*
 * hq.h -- C ABI of libhq.so, the GB300 (sm_103a) state-vector hot path.
 *
 * What the library computes (HybridQ, arXiv 2111.06868):
 *   Sec. 4.2 "State Vector": the evolution engine multiplies each k-qubit gate
 *   (a dense 2^k x 2^k complex matrix, the MatrixGate of Sec. 2) into the
 *   2^n-amplitude state, after Sec. 3.1's compress() has fused neighbouring
 *   gates into blocks of at most max_n_qubits qubits.
 *
 * Conventions (all entry points):
 *   - State: 2^n contiguous interleaved complex amplitudes in DEVICE memory,
 *     complex64 (float re, float im) or complex128 (double re, double im),
 *     16-byte aligned, owned by the caller.  Amplitude index x is the C-order
 *     index of the (2,)*n tensor: qubit q is bit (n-1-q) of x (Sec. 2.2's
 *     Grover printout fixes this order).
 *   - Gate matrix: HOST memory, 2^k x 2^k complex128, row-major, interleaved
 *     (re, im).  Local basis index r = sum_j r_j 2^(k-1-j) with r_j the bit
 *     of qubits[j]: qubits[0] is the most significant (the Kronecker order of
 *     the qubit list, as for MatrixGate(M, qubits)).  The library copies what
 *     it needs before returning; the caller may free it right after.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device work is enqueued asynchronously on it unless
 *     an entry point says it synchronises.
 *   - Errors: every entry point returns hq_status; 0 is success, negative
 *     values are errors.  Arguments are validated on the host before any work
 *     is enqueued; on an argument error nothing is enqueued.  HQ_ERR_CUDA
 *     means a CUDA runtime call failed (text from hq_last_error()).  No C++
 *     exception crosses the boundary.
 *   - Threading: entry points may be called from several host threads; the
 *     per-device library state is set up once under a lock.
 */
#ifndef HQ_H
#define HQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HQ_MAX_K 6      /* widest gate / fused block */
#define HQ_MAX_N 34     /* widest state: 2^34 complex64 = 128 GiB */
#define HQ_MAX_PAULI 8  /* factors per Pauli-string term */

typedef int hq_status;
#define HQ_OK 0
#define HQ_ERR_NULL (-1)         /* a required pointer is NULL */
#define HQ_ERR_QUBIT_RANGE (-2)  /* qubit index outside [0, n) */
#define HQ_ERR_DUP_QUBIT (-3)    /* a qubit repeated within one gate / term */
#define HQ_ERR_K_TOO_LARGE (-4)  /* k < 1 or k > HQ_MAX_K, or k > n */
#define HQ_ERR_N_TOO_LARGE (-5)  /* n < 1 or n > HQ_MAX_N */
#define HQ_ERR_DTYPE (-6)        /* unknown hq_dtype, or dtype not supported by the engine */
#define HQ_ERR_ALLOC (-7)        /* device scratch allocation failed */
#define HQ_ERR_CUDA (-8)         /* a CUDA runtime call failed */
#define HQ_ERR_TIMEOUT (-9)      /* a bounded device-side wait ran out */
#define HQ_ERR_TOKEN (-10)       /* initial-state token not in {0,1,+,-} */
#define HQ_ERR_CAPACITY (-11)    /* an output buffer is too small */
#define HQ_ERR_ARG (-12)         /* any other invalid argument */
#define HQ_ERR_ALIGN (-13)       /* device pointer not 16-byte aligned */

typedef enum { HQ_C64 = 0, HQ_C128 = 1 } hq_dtype;

/* A gate / fused block: k qubits and a host matrix (see conventions). */
typedef struct {
    int k;
    int qubits[HQ_MAX_K];
    const double *matrix;
} hq_gate;

/* One operation of a parametrised circuit (hq_adjoint_grad). */
#define HQ_OP_MATRIX 0 /* fixed gate: k, qubits, matrix as in hq_gate */
#define HQ_OP_ROT 1    /* exp(-i theta P / 2) on qubits[0], P = axis, theta = params[param] */
typedef struct {
    int kind;
    int k;
    int qubits[HQ_MAX_K];
    const double *matrix;
    int axis; /* 'X', 'Y' or 'Z' (HQ_OP_ROT) */
    int param; /* parameter index (HQ_OP_ROT) */
} hq_op;

/* One Pauli-string term coeff * prod_j ops[j]_{qubits[j]}; len = 0 is the identity. */
typedef struct {
    double coeff;
    int len;
    int qubits[HQ_MAX_PAULI];
    char ops[HQ_MAX_PAULI]; /* 'X', 'Y' or 'Z' */
} hq_pauli_term;

/* Kernel choice for hq_apply_blocks. */
#define HQ_ENGINE_AUTO 0      /* cheapest exact path: diagonal / gather / CUDA-core block */
#define HQ_ENGINE_CUDA_CORE 1 /* FP32/FP64 CUDA-core kernels only */
#define HQ_ENGINE_TC_F16 2    /* k >= 5 blocks on tcgen05 tensor cores, FP16 hi+lo split (complex64) */
#define HQ_ENGINE_TC_BF16 3   /* same, BF16 hi+lo split (complex64) */
#define HQ_ENGINE_TC_PASS 4   /* blocks (k <= 6) grouped two at a time into 13-qubit tile passes on tcgen05
                                 tensor cores, FP16 hi+lo split (complex64, n >= 14; smaller n: as TC_F16) */
#define HQ_ENGINE_DF 5        /* complex128 only: diagonal gates and monomial / dense gates of k <= 4 in
                                 double-float arithmetic (48-bit hi + lo float pairs) on the FP32 pipes;
                                 controlled gates and k = 5, 6 blocks as HQ_ENGINE_CUDA_CORE */
#define HQ_ENGINE_TC_C128 6   /* complex128 only: dense k = 3, 4 blocks (n >= 11; k = 3 widened to 4) on
                                 tcgen05 tensor cores as exact FP16 products of 8-bit signed digit slices
                                 (six per operand, FP32 accumulation exact, levels joined in 64-bit
                                 integers); all other gates as HQ_ENGINE_DF */
typedef struct {
    int engine;  /* HQ_ENGINE_* */
    int tc_min_k; /* blocks with k >= tc_min_k use the tensor-core engine (default 5) */
} hq_config;

/* Human-readable name of a status code (static string). */
const char *hq_status_string(hq_status s);
/* Text of the last CUDA error seen by this thread ("" if none). */
const char *hq_last_error(void);
/* Library version string. */
const char *hq_version(void);

/*
 * hq_state_init -- Sec. 4.1 ("Initial and Final State Specification"):
 * write the product state selected by `tokens` (n chars, each '0', '1', '+'
 * or '-'; qubit q takes tokens[q]) into `state`; tokens == NULL gives |0..0>.
 * Device write of 2^n amplitudes on `stream`.
 * Errors: HQ_ERR_NULL (state), HQ_ERR_N_TOO_LARGE, HQ_ERR_DTYPE, HQ_ERR_TOKEN,
 * HQ_ERR_ALIGN, HQ_ERR_CUDA.
 */
hq_status hq_state_init(void *state, int n, hq_dtype dt, const char *tokens, void *stream);

/*
 * hq_state_upload -- copy a state of 2^n amplitudes of type dt from HOST
 * memory `host` (16-byte aligned) into the device state `state` on `stream`,
 * for callers that keep states in host memory (the Sec. 4.2 evolution then
 * runs on the device copy).  Pinned host memory (cudaHostAlloc,
 * cudaHostRegister) is read by the GPU's SMs directly over the CPU-GPU link;
 * other host memory goes through cudaMemcpyAsync.  Asynchronous: the host
 * buffer must stay valid and unchanged until the stream has passed this
 * point.  Not in the paper.
 * Errors: HQ_ERR_NULL, HQ_ERR_N_TOO_LARGE, HQ_ERR_DTYPE, HQ_ERR_ALIGN (either
 * pointer), HQ_ERR_CUDA.
 */
hq_status hq_state_upload(void *state, const void *host, int n, hq_dtype dt, void *stream);

/*
 * hq_fuse -- Sec. 3.1 compress(circuit, max_n_qubits): greedily merge the G
 * gates (host) into blocks of at most k_max qubits (1 <= k_max <= HQ_MAX_K).
 * A gate joins the latest earlier block that shares a qubit with it when the
 * union fits; otherwise the earliest later block (all of them disjoint from
 * the gate, so the move commutes) whose union fits; otherwise it opens a new
 * block.  Each block's qubits are sorted ascending and its matrix is the
 * product of its members (later members on the left), embedded in that order,
 * computed in double on the host.
 *   blocks:     out, capacity *B on entry; *B = number of blocks on return.
 *   pool:       out, host doubles receiving the block matrices (blocks[i].matrix
 *               points into it); pool_len = its capacity in doubles.  Worst case
 *               is G * 2 * 4^k_max.
 *   gate_block: optional out (G ints): the block index of every gate.
 * Host only; no device work.  Errors: HQ_ERR_NULL, HQ_ERR_ARG (k_max, G < 0),
 * HQ_ERR_K_TOO_LARGE (a gate wider than k_max), HQ_ERR_QUBIT_RANGE,
 * HQ_ERR_DUP_QUBIT, HQ_ERR_CAPACITY (blocks or pool too small).
 */
hq_status hq_fuse(int n, const hq_gate *gates, int G, int k_max, hq_gate *blocks, int *B, double *pool,
                  int64_t pool_len, int *gate_block);

/*
 * hq_fuse_dag -- Sec. 3.1 compress(circuit, max_n_qubits) with a different
 * rule: the same output as hq_fuse (blocks of at most k_max qubits, qubits
 * sorted ascending, matrix = product of the members, FP64 on the host), in
 * usually fewer blocks.  The circuit is read as a DAG (gates keep their order
 * on every qubit, which fixes the product).  Blocks are placed one at a time
 * from the DAG frontier: from each frontier gate a qubit set is grown one
 * qubit at a time, each time by the qubit that lets the block absorb the most
 * frontier gates inside the set (3 points per multi-qubit gate, 1 per
 * single-qubit gate), and the best such block is placed.  A final pass merges
 * a block into an earlier or later one when every block in between shares no
 * qubit with it and the union fits.
 *   restarts: >= 1 runs; run 0 breaks ties by the lowest index, run r > 0 at
 *             random from SplitMix64 seeded with seed + r; the run with the
 *             fewest blocks is returned (the first of equal runs).
 *   other arguments, ownership and errors: as hq_fuse (restarts < 1: HQ_ERR_ARG).
 * Host only; no device work.  Cost: about restarts x (a few ms per 1000
 * gates).
 */
hq_status hq_fuse_dag(int n, const hq_gate *gates, int G, int k_max, int restarts, uint64_t seed,
                      hq_gate *blocks, int *B, double *pool, int64_t pool_len, int *gate_block);

/*
 * hq_fuse_beam -- Sec. 3.1 compress(circuit, max_n_qubits) by a beam search
 * over the block sequences of hq_fuse_dag: the same output (blocks of at most
 * k_max qubits, qubits ascending, matrix = product of the members in FP64),
 * in as few or fewer blocks.  Each step extends every one of the `width`
 * kept sequences by one block (proposed from each frontier gate by the
 * hq_fuse_dag growth rule, once with the lowest-index tie-break and three
 * times with SplitMix64 tie-breaks seeded from seed, the step and the
 * sequence), keeps the `width` extensions that have absorbed the most gates
 * (3 points per multi-qubit gate, 1 per single-qubit gate; one per distinct
 * DAG frontier), and stops at the first sequence that absorbs every gate;
 * hq_fuse_dag's merge pass follows.  The result is never worse than
 * hq_fuse_dag's first run, and the same for the same arguments on any host.
 *   width: 1..4096 kept sequences.
 *   other arguments, ownership and errors: as hq_fuse (width out of range:
 *   HQ_ERR_ARG).
 * Host only; no device work; spreads the sequences over up to 16 host
 * threads.  Cost: about width x (a few ms per 1000 gates) of CPU time.
 */
hq_status hq_fuse_beam(int n, const hq_gate *gates, int G, int k_max, int width, uint64_t seed,
                       hq_gate *blocks, int *B, double *pool, int64_t pool_len, int *gate_block);

/*
 * hq_reduced_density_matrix -- the reduced density matrix of k <= 2 qubits
 * of a pure state: rho_ab = sum over the other qubits' indices y of
 * psi(y, a) conj(psi(y, b)), a and b local indices with qubits[0] as MSB
 * (Sec. 5; the one-qubit case is the paper's noisy tensor-network example).
 * One read of the state, FP64 sums; synchronous.
 *   rho_host: out, 2 * 4^k doubles, row-major complex.
 * Errors: HQ_ERR_NULL, HQ_ERR_N_TOO_LARGE, HQ_ERR_DTYPE, HQ_ERR_ALIGN,
 * HQ_ERR_K_TOO_LARGE (k < 1 or k > 2), HQ_ERR_QUBIT_RANGE, HQ_ERR_DUP_QUBIT,
 * HQ_ERR_ALLOC, HQ_ERR_CUDA.
 */
hq_status hq_reduced_density_matrix(const void *state, int n, hq_dtype dt, const int *qubits, int k,
                                    double *rho_host, void *stream);

/*
 * hq_apply_kraus_sampled -- Sec. 5 pure-state sampling of the Kraus
 * operators K_0..K_{nK-1} of a channel on k <= 2 qubits: p_i = ||K_i psi||^2
 * (from the operators alone when every K_i^dag K_i is a multiple of the
 * identity, e.g. Pauli channels; else Tr(K_i rho K_i^dag) from the
 * reduced density matrix, on the device), i = the first index whose
 * cumulative probability exceeds u * sum p, then psi <- K_i psi / sqrt(p_i).
 *   kraus:  nK matrices of 2^k x 2^k complex128, row-major, one after another.
 *   u:      a uniform number in [0, 1) drawn by the caller.
 *   chosen: out (may be NULL), the index i.
 * Errors: as hq_reduced_density_matrix, plus HQ_ERR_ARG (nK outside
 * [1, 64], u outside [0, 1), or every p_i = 0).
 */
hq_status hq_apply_kraus_sampled(void *state, int n, hq_dtype dt, const int *qubits, int k, int nK,
                                 const double *kraus, double u, int *chosen, void *stream);

/* one operation of a noisy circuit (hq_run_trajectory) */
typedef struct {
    int k;               /* qubits acted on: 1..HQ_MAX_K for gates, 1..2 for channels */
    int qubits[HQ_MAX_K];
    int nkraus;          /* 0: a gate (matrix = one 2^k x 2^k matrix); >= 1: a channel with nkraus Kraus operators */
    const double *matrix; /* complex128, row-major, host; nkraus matrices one after another for a channel */
} hq_noisy_op;

/*
 * hq_run_trajectory -- one pure-state trajectory of a noisy circuit (Sec. 5):
 * gates applied as hq_apply_blocks applies them (engine from cfg, NULL =
 * HQ_ENGINE_AUTO), each channel as hq_apply_kraus_sampled with the next
 * entry of u.
 *   u:      one uniform in [0, 1) per channel, in operation order.
 *   chosen: out (may be NULL), the sampled Kraus index per channel.
 * Channels whose operators all have K_i^dag K_i = p_i I are sampled on the
 * host from p_i alone; the others on the device (reduced density matrix,
 * branch and renormalised operator picked by one CTA, no host round trip).
 * The operators applied right before a device-sampled channel on the same
 * qubits, in the same order, are folded into it (probabilities from
 * A rho A^dag, K_i A / sqrt(p_i) applied): the same result in fewer passes.
 * Synchronous once, at the end, when a channel was sampled on the device;
 * device scratch (operators, partial sums) from the stream-ordered
 * allocator, released before returning.
 * Errors: as hq_apply_gate and hq_apply_kraus_sampled; HQ_ERR_ARG (nops < 0).
 */
hq_status hq_run_trajectory(void *state, int n, hq_dtype dt, const hq_noisy_op *ops, int nops, const double *u,
                            int *chosen, const hq_config *cfg, void *stream);

/*
 * Density matrices -- Sec. 5 ("Simulations with noise"): exact evolution of
 * rho under maps Lambda[X] = sum_ij s_ij L_i X R_j^dag (Sec. 2's
 * KrausSuperGate), each applied, as Sec. 2's MatrixSuperGate does, as one
 * matrix-vector product on the vectorised rho.
 * Layout: rho (2^n x 2^n) is the 2n-qubit state vector vec(rho), row-major:
 * entry (x, y) at flat index x 2^n + y, so (in the state-vector conventions
 * above) qubit q of the row index is vector qubit q and qubit q of the
 * column index is vector qubit n + q.  4^n complex entries in DEVICE memory,
 * complex64 or complex128, 16-byte aligned, caller-owned; 1 <= n <= 17.
 * The map of a k-qubit operation is the 2k-qubit gate
 *   S = sum_ij s_ij L_i (x) conj(R_j)   (row-major vec(A X B) = (A (x) B^T) vec X)
 * on vector qubits (q_0..q_{k-1}, n+q_0..n+q_{k-1}): its pair index is
 * a 2^k + b for the local row index a and column index b (qubits[0] the most
 * significant bit of each).
 */
#define HQ_DM_MAX_K 3      /* widest operation: its superoperator spans 2k <= HQ_MAX_K vector qubits */
#define HQ_DM_MAX_OPS 4096 /* most left (or right) operators of one map */
#define HQ_DM_MAP 0        /* Lambda[rho] = sum_ij s_ij L_i rho R_j^dag (KrausSuperGate) */
#define HQ_DM_SUPER 1      /* a 4^k x 4^k superoperator matrix on the pair index (MatrixSuperGate) */
typedef struct {
    int kind;             /* HQ_DM_MAP or HQ_DM_SUPER */
    int k;                /* 1..HQ_DM_MAX_K */
    int qubits[HQ_DM_MAX_K];
    int nl, nr;           /* HQ_DM_MAP: numbers of left and right operators */
    const double *left;   /* HQ_DM_MAP: nl matrices 2^k x 2^k, one after another; HQ_DM_SUPER: the
                             4^k x 4^k matrix.  complex128, row-major, host */
    const double *right;  /* HQ_DM_MAP: nr matrices, or NULL for R = L (nr ignored) */
    const double *s;      /* HQ_DM_MAP: nl x nr complex128 coefficients, row-major, or NULL for the
                             identity (needs nl == nr) */
} hq_dm_op;
/* A unitary gate U: HQ_DM_MAP, nl = 1, left = U, right = s = NULL (rho -> U rho U^dag).
   A Kraus channel {K_i}: HQ_DM_MAP, nl = number of operators, right = s = NULL. */

/*
 * hq_dm_superop -- the superoperator S of a map (host, FP64; see above):
 * S_out receives 2 * 16^k doubles (4^k x 4^k complex, row-major).
 * Errors: HQ_ERR_NULL, HQ_ERR_K_TOO_LARGE (k outside [1, HQ_DM_MAX_K]),
 * HQ_ERR_ARG (nl or nr outside [1, HQ_DM_MAX_OPS]; s == NULL with nr != nl).
 */
hq_status hq_dm_superop(int k, int nl, const double *left, int nr, const double *right, const double *s,
                        double *S_out);

/*
 * hq_dm_init -- rho = |psi0><psi0| for the product state of hq_state_init's
 * tokens (NULL: |0..0><0..0|); written as the 2n-qubit product state with
 * the tokens repeated (the token amplitudes are real).  Device write of 4^n
 * entries on `stream`.  Errors: as hq_state_init (n outside [1, 17]:
 * HQ_ERR_N_TOO_LARGE).
 */
hq_status hq_dm_init(void *rho, int n, hq_dtype dt, const char *tokens, void *stream);

/*
 * hq_dm_apply -- rho <- Lambda_nops ... Lambda_1 [rho] exactly (the density-
 * matrix level of Sec. 5).  Every operation becomes its superoperator (host,
 * FP64); with k_max >= 2 they are fused by hq_fuse_dag into blocks of at most
 * k_max vector qubits (8 seeded runs, seed 0); k_max = 0 applies one block per
 * operation.  The blocks run through hq_apply_blocks with cfg (NULL =
 * HQ_ENGINE_AUTO) on the 2n-qubit vector, asynchronously on `stream`.
 * Errors: as hq_dm_init and hq_apply_blocks; HQ_ERR_ARG (nops < 0, k_max
 * outside [0, HQ_MAX_K], unknown kind, operator counts as hq_dm_superop),
 * HQ_ERR_K_TOO_LARGE (an operation with 2k > k_max > 0), HQ_ERR_QUBIT_RANGE,
 * HQ_ERR_DUP_QUBIT.
 */
hq_status hq_dm_apply(void *rho, int n, hq_dtype dt, const hq_dm_op *ops, int nops, int k_max, const hq_config *cfg,
                      void *stream);

/*
 * hq_dm_expectation -- Tr(rho H) = sum_t coeff_t sum_x rho[x][x ^ m_t] P_t[x ^ m_t][x]
 * for a Pauli sum (hq_pauli_term, as hq_expectation; len 0 gives Tr rho),
 * the real part, accumulated in double: reads 2^n of the 4^n entries per
 * term.  SYNCHRONISES `stream`; device scratch (per-CTA partial sums) from
 * the stream-ordered allocator, released before returning.
 * Errors: as hq_expectation (n outside [1, 17]: HQ_ERR_N_TOO_LARGE).
 */
hq_status hq_dm_expectation(const void *rho, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                            double *out_host, void *stream);

/*
 * hq_dm_purity -- Tr(rho^2) = sum_xy |rho_xy|^2 for a Hermitian rho (the
 * squared norm of vec(rho), as hq_expectation computes it).  SYNCHRONISES
 * `stream`.  Errors: as hq_dm_expectation.
 */
hq_status hq_dm_purity(const void *rho, int n, hq_dtype dt, double *out_host, void *stream);

/*
 * hq_pop -- Sec. 3.1 pop(circuit, pinned_qubits): mark the gates inside the
 * light cone of the pinned qubits (host only).  HQ_POP_RIGHT walks from the
 * last gate back: a gate is kept when it shares a qubit with the cone, whose
 * qubits then join the cone; the gates dropped act, after every kept gate
 * that touches their qubits, on qubits that never reach the pinned ones, so
 * the reduced state of the pinned qubits (and every expectation value of an
 * observable on them) is unchanged.  HQ_POP_LEFT walks from the first gate
 * forward (the same for the inverse circuit).  Matrices are not read (may be
 * NULL).
 *   pinned: npinned qubit indices (repeats allowed).
 *   keep:   out, G ints: 1 = kept, 0 = dropped.
 * Returns the number of kept gates, or HQ_ERR_NULL, HQ_ERR_ARG (G < 0,
 * npinned < 0, direction), HQ_ERR_N_TOO_LARGE (n outside [1, 64]),
 * HQ_ERR_QUBIT_RANGE, HQ_ERR_K_TOO_LARGE, HQ_ERR_DUP_QUBIT.
 */
#define HQ_POP_RIGHT 0
#define HQ_POP_LEFT 1
int hq_pop(int n, const hq_gate *gates, int G, const int *pinned, int npinned, int direction, int *keep);

/*
 * hq_simplify -- Sec. 3.1 simplify(circuit, use_matrix_commutation): mark
 * the gates that remain after dropping (host only, FP64)
 *   - every gate within atol of the identity (max-abs over its entries), and
 *   - pairs g < h on the same qubit set whose product h g is within atol of
 *     the identity, where h commutes with every kept gate between them that
 *     shares a qubit with it: by having no qubit in common, or, with
 *     use_matrix_commutation, by |[A, B]| <= atol on the union of their qubits
 *     (unions wider than 8 qubits count as not commuting).
 * Pairs are removed until none is left.  The kept gates, in their order, give
 * the same operator within the tolerances.
 *   keep: out, G ints: 1 = kept, 0 = dropped.
 * Returns the number of kept gates, or HQ_ERR_NULL, HQ_ERR_ARG (G < 0, atol
 * negative or NaN), HQ_ERR_N_TOO_LARGE (n outside [1, 64]),
 * HQ_ERR_QUBIT_RANGE, HQ_ERR_K_TOO_LARGE, HQ_ERR_DUP_QUBIT.
 */
int hq_simplify(int n, const hq_gate *gates, int G, int use_matrix_commutation, double atol, int *keep);

/*
 * hq_gate_structure -- the structure hq_apply_gate looks for in a k-qubit
 * matrix (complex128, row-major as in hq_gate; host only, no device work).
 * Returns a bit set (>= 0) of
 *   HQ_STRUCT_DIAGONAL   every off-diagonal entry exactly 0;
 *   HQ_STRUCT_MONOMIAL   one nonzero per row and column (entries within
 *                        4 FP64 epsilon of the largest magnitude count as 0);
 *   HQ_STRUCT_CONTROLLED at least one control (Sec. 2's Control gates): the
 *                        matrix is the identity on every row and column where
 *                        that qubit is 0 (same tolerance);
 * or HQ_ERR_NULL (matrix) / HQ_ERR_K_TOO_LARGE (k out of [1, HQ_MAX_K]).
 *   control_mask: optional out; bit j set when qubits[j] is a control.
 *   u: optional out, 2 * 4^kt doubles for kt = k - (number of controls): the
 *      matrix on the remaining targets (in their order, first = MSB of the
 *      local index) where every control is 1.
 */
#define HQ_STRUCT_DIAGONAL 1
#define HQ_STRUCT_MONOMIAL 2
#define HQ_STRUCT_CONTROLLED 4
int hq_gate_structure(int k, const double *matrix, int *control_mask, double *u);

/*
 * hq_apply_gate -- Sec. 4.2: state <- (matrix on qubits[0..k-1]) state, for
 * every group of 2^k amplitudes that differ only in the target bits.  Picks a
 * kernel from the matrix's structure and the target positions: controlled
 * gates with at most 2 targets and a control above the 32-byte sector read
 * and write only the amplitudes whose controls are all 1; then diagonal
 * gates a stream over the state; monomial gates (k <= 4) a permuted, phased
 * copy; dense k <= 4 the shared-memory gather kernel; k = 5, 6 the CUDA-core
 * block kernel.
 * Errors: HQ_ERR_NULL, HQ_ERR_N_TOO_LARGE, HQ_ERR_K_TOO_LARGE,
 * HQ_ERR_QUBIT_RANGE, HQ_ERR_DUP_QUBIT, HQ_ERR_DTYPE, HQ_ERR_ALIGN,
 * HQ_ERR_ALLOC, HQ_ERR_CUDA.
 */
hq_status hq_apply_gate(void *state, int n, hq_dtype dt, const int *qubits, int k, const double *matrix,
                        void *stream);

/*
 * hq_apply_blocks -- apply G gates / fused blocks in order (the evolution
 * loop of Sec. 4.2), choosing a kernel per block as configured (cfg NULL =
 * HQ_ENGINE_AUTO).  Tensor-core engines apply only to complex64 states,
 * HQ_ENGINE_DF and HQ_ENGINE_TC_C128 only to complex128 states (HQ_ERR_DTYPE
 * otherwise).
 * HQ_ENGINE_TC_PASS applies the same operators in the same order (blocks
 * with disjoint targets may swap), up to two per read and write of the state:
 * see hq_plan_passes.  It moves qubits between bit positions while it runs and
 * restores the caller's order before it returns (stream order).
 * Errors: as hq_apply_gate, plus HQ_ERR_ARG (G < 0 or unknown engine).
 * On HQ_ERR_ALLOC the state is left as follows: the tensor-core engines and
 * HQ_ENGINE_TC_PASS take their one scratch buffer before enqueueing any
 * kernel, so the state is untouched; HQ_ENGINE_AUTO / HQ_ENGINE_CUDA_CORE
 * allocate per wide (k = 5, 6) block, so the blocks before the one whose
 * allocation failed have been applied and none after it.
 */
hq_status hq_apply_blocks(void *state, int n, hq_dtype dt, const hq_gate *gates, int G, const hq_config *cfg,
                          void *stream);

/*
 * hq_simulate -- Sec. 4.2 simulate(circuit, initial_state): state <- the
 * gates / fused blocks applied in order (as hq_apply_blocks applies them with
 * cfg) to the Sec. 4.1 product state of `tokens` (as hq_state_init; NULL =
 * |0..0>); with norm2_host set, also the squared norm sum |psi_x|^2 of the
 * result, accumulated in double.  The same result as hq_state_init,
 * hq_apply_blocks and hq_expectation of the identity in a row, in fewer
 * passes over the state on the tensor-core engines (complex64, n >= 13): a first
 * block that runs on the tensor cores computes its input amplitudes from the
 * tokens instead of reading an initialised state, and a last one that does
 * sums |psi_x|^2 of what it writes (FP32 within a tile, in chains of at
 * most 16 squares, FP64 across tiles, the per-warp sums added on the host in
 * a fixed order: within 1e-8 relative of the exact sum of the stored
 * amplitudes).  With norm2_host set, a last block of 4..6 qubits that a
 * structured kernel would take (diagonal, monomial, controlled) runs on the
 * tensor cores as well, so that it sums the norm: its result then carries
 * the split-precision rounding instead of being exact in FP32.  Other
 * engines and blocks run the separate passes.
 *   state: out, 2^n amplitudes (DEVICE, caller-owned, 16-byte aligned); its
 *          previous contents are never read.
 *   norm2_host: out (may be NULL); when set the call SYNCHRONISES `stream`
 *          and reports a device-side timeout as HQ_ERR_TIMEOUT; when NULL it
 *          only enqueues work.
 * Device scratch (split matrices, per-warp norm sums) from the stream-ordered
 * allocator, released before returning.
 * Errors: as hq_state_init and hq_apply_blocks; HQ_ERR_TIMEOUT.
 */
hq_status hq_simulate(void *state, int n, hq_dtype dt, const char *tokens, const hq_gate *gates, int G,
                      const hq_config *cfg, double *norm2_host, void *stream);

/*
 * hq_plan_passes -- the plan HQ_ENGINE_TC_PASS executes for these gates (for
 * inspection and tests).  A pass holds a tile of 13 physical bit positions
 * that includes bits 0..6, applies up to max_blocks (1 or 2) of the gates to
 * it in order, and moves the qubit at each of its positions to another of
 * them; passes with no gate only move qubits (the final ones restore the
 * caller's order).  Physical bit x initially holds qubit n-1-x.
 *   records: out, max_passes records of HQ_PASS_RECORD ints each:
 *            slots[13] (ascending), nb, gate[2] (indices into gates, -1
 *            unused), dest[13] (new position of the qubit at slots[j]).
 * Returns the number of passes (which may exceed max_passes: then only the
 * first max_passes are written), or a negative hq_status: HQ_ERR_NULL,
 * HQ_ERR_ARG (n < 14 or > 40, G < 0, max_blocks not 1 or 2),
 * HQ_ERR_K_TOO_LARGE (k > 6), HQ_ERR_QUBIT_RANGE, HQ_ERR_DUP_QUBIT.
 * Host only; no device work.
 */
#define HQ_PASS_RECORD 29
int hq_plan_passes(int n, const hq_gate *gates, int G, int max_blocks, int *records, int max_passes);

/*
 * hq_test_fail_next_allocs -- fault injection for tests of the error paths
 * (no counterpart in the paper): the next `count` device scratch allocations
 * the library takes from the stream-ordered allocator (hq_expectation,
 * hq_reduced_density_matrix, the channel sampling of hq_apply_kraus_sampled
 * and hq_run_trajectory, hq_dm_expectation, and the matrix buffers of the
 * CUDA-core wide blocks, the tensor-core engines and the tile-pass engine of
 * hq_apply_blocks) fail as if the device were out of
 * memory; the entry point that meets one returns HQ_ERR_ALLOC (work it had
 * enqueued before stays enqueued).  count = 0 turns it off.  Process-wide;
 * host only.  Errors: HQ_ERR_ARG (count < 0).
 */
hq_status hq_test_fail_next_allocs(int count);

/*
 * hq_expectation -- <psi|H|psi> = sum_t coeff_t <psi|P_t|psi> for a Pauli sum
 * (T terms), accumulated in double; a term of len 0 gives the squared norm.
 * Result written to *out_host.  SYNCHRONISES `stream`.  Uses device scratch
 * (per-block partial sums, a few hundred KB) from the stream-ordered
 * allocator, released before returning.
 * Errors: HQ_ERR_NULL, HQ_ERR_N_TOO_LARGE, HQ_ERR_DTYPE, HQ_ERR_QUBIT_RANGE,
 * HQ_ERR_DUP_QUBIT, HQ_ERR_ARG (len out of [0, HQ_MAX_PAULI], bad op char,
 * T < 0), HQ_ERR_ALIGN, HQ_ERR_ALLOC, HQ_ERR_CUDA.
 */
hq_status hq_expectation(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                         double *out_host, void *stream);

/*
 * hq_expectation_static -- the same result as hq_expectation, computed
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (or any
 * allocator) at the point of the call -- for example a host that hands all
 * device memory to its own pool up front, a serving loop that forbids
 * allocator calls for predictable latency, or code that must not allocate
 * while another component is capturing or replaying work on the device.
 *
 * The per-block partial sums live in a file-scope device array of
 * 64 x 512 + 1 doubles (256 KiB + 8 bytes) that every GPU which loads
 * libhq.so keeps until the process exits.  Limits: at most 64 X-mask groups
 * after splitting (terms that share their X/Y positions form one group; a
 * group holds at most 48 terms), otherwise HQ_ERR_CAPACITY with the reason
 * in hq_last_error(); every other argument rule is that of hq_expectation.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it: make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents;
 * each call writes every slot it reads, so no clearing is needed, but calls
 * whose work overlaps on the GPU (different streams or host threads) race on
 * it and must be serialised by the caller.  Result written to *out_host;
 * SYNCHRONISES `stream`.
 */
hq_status hq_expectation_static(const void *state, int n, hq_dtype dt, const hq_pauli_term *terms, int T,
                                double *out_host, void *stream);

/*
 * hq_adjoint_workspace_bytes -- device workspace hq_adjoint_grad needs for
 * `batch` parameter sets of an n-qubit, G-operation, P-parameter circuit
 * with `checkpoints` stored forward states per parameter set (0 = none).
 */
size_t hq_adjoint_workspace_bytes(int n, hq_dtype dt, int G, int P, int batch, int checkpoints);

/*
 * hq_adjoint_grad -- energy E_b = <psi_b|H|psi_b>, psi_b = U(theta_b)|tokens>,
 * and its gradient dE_b/dtheta_b[p] for every parameter, for `batch`
 * parameter sets (theta_host: batch x P doubles, row-major).  Not in the
 * paper: the adjoint reverse sweep (Jones & Gacon, arXiv 2009.02823) with two
 * state vectors per parameter set.  The reverse sweep recomputes earlier
 * states by applying U^+; with checkpoints > 0 it also stores that many
 * evenly spaced forward states and restores them on the way back.
 *   workspace: caller-owned device memory of at least
 *              hq_adjoint_workspace_bytes(...) bytes (ws_bytes).
 *   energies_host: out, batch doubles.  grads_host: out, batch x P doubles.
 * SYNCHRONISES `stream`.  Errors: as hq_apply_gate and hq_expectation, plus
 * HQ_ERR_ARG (kind/axis/param out of range, batch < 1), HQ_ERR_CAPACITY
 * (ws_bytes too small).
 */
hq_status hq_adjoint_grad(int n, hq_dtype dt, const hq_op *ops, int G, int P, const double *theta_host,
                          int batch, const hq_pauli_term *H, int T, const char *tokens, int checkpoints,
                          void *workspace, size_t ws_bytes, double *energies_host, double *grads_host,
                          void *stream);

/*
 * Batched runs -- many independent circuits of uneven size in ONE persistent
 * kernel launch, captured once into a CUDA graph and replayed (serving-style
 * loads).  Not in the paper beyond its evolution of each circuit (Sec. 4.2)
 * and its gate grouping (Sec. 3.1): every circuit starts from |0..0> and its
 * gates (k <= 2, host matrices) are grouped into passes; one pass = one read
 * and one write of the state, during which each tile of 2^tile_bits
 * amplitudes (the lowest tile_bits - max_high bits as one contiguous run, plus
 * up to max_high higher bits) stays in shared memory while the pass's gates
 * are applied.  A circuit with n <= tile_bits is one pass over one tile.
 */
typedef struct {
    int n;                /* qubits, 1..30 */
    int G;                /* gates */
    const hq_gate *gates; /* host; each k <= 2 */
    void *state;          /* device, 2^n complex64, 16-byte aligned, caller-owned; overwritten */
} hq_circuit;

typedef struct {
    int tile_bits;   /* log2 amplitudes per shared-memory tile, 6..13 (0 = 12) */
    int max_high;    /* high bits per pass, 1..8, < tile_bits (0 = 6) */
    int ctas_per_sm; /* persistent CTAs per SM (0 = as many as fit) */
    int small_first; /* queue circuits smallest first (lower median latency) instead of largest first */
    int fuse_k;      /* width of the blocks a pass's gates are fused into (Sec. 3.1 compress), 1..3 (0 = 2) */
} hq_batch_config;

typedef struct hq_batch hq_batch; /* opaque plan + instantiated CUDA graph */

/* Device workspace hq_batch_create needs for this batch (0 on invalid input). */
size_t hq_batch_workspace_bytes(const hq_circuit *cs, int C, const hq_batch_config *cfg);

/*
 * hq_batch_create -- validate, plan (host), upload the plan into `workspace`
 * (caller-owned device memory of >= hq_batch_workspace_bytes bytes, 256-byte
 * aligned) and capture the run (counter reset + persistent kernel) into a CUDA
 * graph.  SYNCHRONISES `stream`.  The circuits' gates are copied; their state
 * buffers and the workspace must outlive the handle.
 * Errors: HQ_ERR_NULL, HQ_ERR_ARG (C < 1, bad config), HQ_ERR_N_TOO_LARGE,
 * HQ_ERR_K_TOO_LARGE (a gate with k > 2), HQ_ERR_QUBIT_RANGE,
 * HQ_ERR_DUP_QUBIT, HQ_ERR_ALIGN, HQ_ERR_CAPACITY, HQ_ERR_CUDA.
 */
hq_status hq_batch_create(const hq_circuit *cs, int C, const hq_batch_config *cfg, void *workspace, size_t ws_bytes,
                          void *stream, hq_batch **out);

/* hq_batch_run -- enqueue one replay of the captured graph on `stream` (async):
 * every circuit's state is rebuilt from |0..0> and evolved. */
hq_status hq_batch_run(hq_batch *b, void *stream);

/*
 * hq_batch_latencies -- after a run on `stream` (SYNCHRONISES it): completion
 * time of each circuit (latency_us, C floats, may be NULL) and of the whole
 * batch (makespan_us), in microseconds since the kernel started.  Returns
 * HQ_ERR_TIMEOUT if the run stopped because its bounded scheduler wait ran
 * out (2 s without progress).
 */
hq_status hq_batch_latencies(hq_batch *b, void *stream, float *latency_us, double *makespan_us);

/*
 * hq_test_batch_wait_limit_ns -- for tests of the bounded-wait path (no
 * counterpart in the paper).  The batch runner's scheduler gives up, raises
 * the device error flag and ends its CTA once it has searched for `ns`
 * nanoseconds without finding a tile it may run; the next hq_batch_latencies
 * (or any other entry point that reads the flag) then returns HQ_ERR_TIMEOUT
 * and clears it.  The default limit is 2 s; ns = 0 restores it.  The limit
 * is a device variable of the current device, read by every launch of the
 * runner from then on (graphs already instantiated included); set it while
 * no batch run is in flight.  A run that gave up leaves its states partly
 * evolved; the next run starts them again from |0..0>.
 * Errors: HQ_ERR_CUDA.
 */
hq_status hq_test_batch_wait_limit_ns(unsigned long long ns);

/* hq_batch_destroy -- release the graph and the handle (not the workspace). */
void hq_batch_destroy(hq_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* HQ_H */
