/*
 * tt.h -- C ABI of the GB300 TT-arithmetic library (libttgb.so).
 *
 * Operations follow the problem statements of Al Daas, Ballard, Benner,
 * "Parallel Algorithms for Tensor Train Arithmetic" (arXiv 2011.06532):
 *   tt_round     Alg. 2 / Alg. 6 (TT rounding)
 *   tt_add       Sec. 3.2.1 (summation)
 *   tt_hadamard  Sec. 3.2.2 (Hadamard product)
 *   tt_dot       Sec. 3.2.3, Eq. innerprodsum (inner product)
 *   tt_norm      Sec. 3.2.4 (norm through orthonormalization)
 *   tt_orthonormalize  Alg. 1 / Alg. 5 and the left-hand mirror (Sec. 3.4)
 *   tt_round_ordered   the RLR and LRL orderings of rounding (Sec. 3.4, 4.3.2)
 *   tt_round_sharded   rounding of a tensor distributed over shards (Sec. 3.1, 3.3)
 *
 * Tensor layout.  A TT tensor X has N >= 1 cores; core n (0-based) is an
 * R[n] x I[n] x R[n+1] array with R[0] = R[N] = 1 (Sec. 2.1).  Entry (a, i, b)
 * of core n is element a + R[n] * (i + I[n] * b) of that core's buffer: the
 * "vec-oriented" order of Sec. 3.1, in which the horizontal unfolding H
 * (R[n] x I[n]R[n+1]) and the vertical unfolding V (R[n]I[n] x R[n+1]) of
 * Sec. 2.2 are both column-major.  Core buffers live in device memory of the
 * current CUDA device.
 *
 * Element type and precision.  dtype TT_F64 (TT_PREC_FP64): every step
 * computes in FP64.  dtype TT_F32: cores are stored and streamed in FP32; the
 * per-slab work (push, Householder QR and its applications) runs on the FP32
 * pipes either in double-float arithmetic (TT_PREC_FP32X2: each value an
 * unevaluated sum of two FP32 numbers, about 2^-46 relative accuracy) or in
 * plain FP32 (TT_PREC_FP32); the small factors (triangular-factor reduction
 * trees, SVDs, rank choice, norm) stay in FP64; the result is stored in FP32.
 *
 * Ownership.  The library never allocates memory.  Inputs are borrowed and
 * never modified.  Outputs are caller-owned device buffers.  Routines that need
 * scratch space take a caller-owned device workspace whose size the matching
 * *_workspace_size query returns; the workspace must stay untouched until the
 * work queued on the stream has finished.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 * queued on it.  tt_round, tt_dot and tt_norm synchronize the stream before
 * returning because they return host values (ranks, scalars).
 *
 * Errors.  Every routine returns a tt_status.  On TT_ERR_INVALID_ARG nothing
 * is queued.  On any error the output contents are unspecified.  Routines are
 * deterministic: the same input on the same GPU gives the same bits.
 */
#ifndef TTGB_TT_H
#define TTGB_TT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_ERR_INVALID_ARG = 1, /* bad shape, rank, eps, dtype, null pointer or mode-size mismatch */
  TT_ERR_WORKSPACE = 2,   /* workspace missing or smaller than the size query returned */
  TT_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  TT_ERR_NUMERICAL = 4,   /* non-finite values met, or an SVD did not converge */
  TT_ERR_UNSUPPORTED = 6, /* a rank above TT_MAX_RANK, or a shape whose buffers the
                             planner cannot place */
  TT_ERR_COMM = 7         /* the all-gather callback of a sharded call failed */
} tt_status;

typedef enum { TT_F64 = 0, TT_F32 = 1 } tt_dtype;

typedef enum {
  TT_PREC_DEFAULT = 0, /* TT_PREC_FP64 for TT_F64 cores, TT_PREC_FP32X2 for TT_F32 cores */
  TT_PREC_FP64 = 1,    /* TT_F64 cores only */
  TT_PREC_FP32X2 = 2,  /* TT_F32 cores: double-float slab arithmetic, FP64 small factors */
  TT_PREC_FP32 = 3     /* TT_F32 cores: FP32 slab arithmetic, FP64 small factors */
} tt_precision;

/* Largest rank (R[n]) any routine accepts. */
#define TT_MAX_RANK 160

typedef struct {
  int32_t N;            /* number of cores, >= 1 */
  int32_t dtype;        /* tt_dtype; all cores share it */
  const int64_t *I;     /* host array [N], mode sizes, each >= 1 */
  int64_t *R;           /* host array [N+1], ranks, R[0] = R[N] = 1, each >= 1;
                           written by routines that produce this tensor */
  void *const *cores;   /* host array [N] of pointers the current device can
                           dereference (its own memory, managed memory, or mapped
                           page-locked host memory; any other pointer makes a compute
                           routine return TT_ERR_INVALID_ARG before queueing work),
                           core n holds R[n] * I[n] * R[n+1] elements of dtype */
} tt_tensor;

/*
 * Workspace bytes tt_round needs for input x at `precision` (a tt_precision;
 * depends on N, I, R, dtype and precision only).
 */
int tt_round_workspace_size(const tt_tensor *x, int precision, size_t *bytes);

/*
 * TT rounding (Alg. 2, organised as Alg. 6): a right-to-left sweep takes a
 * tall-skinny QR of every H(X_n)^T (n = N..2) and pushes the triangular factor
 * into core n-1; ||X|| is then the Frobenius norm of the first core; a
 * left-to-right sweep takes, for n = 1..N-1, the SVD of the R factor of V(Y_n),
 * keeps the smallest L_n with sum_{j > L_n} sigma_j^2 <= delta^2, delta =
 * eps ||X|| / sqrt(N-1), writes the column-orthonormal core Q U(:, 1:L_n) and
 * passes Sigma V^T on.  The result Y satisfies ||X - Y|| <= eps ||X|| (Alg. 2).
 *
 * x      input tensor (read only).
 * eps    relative accuracy, finite and >= 0.
 * precision  a tt_precision matching x->dtype (TT_PREC_DEFAULT picks it).
 * out    out->N, out->dtype and out->I must match x; out->cores[n] must hold at
 *        least x->R[n] * I[n] * x->R[n+1] elements (ranks never grow).  On
 *        return out->R holds the new ranks and core n holds
 *        out->R[n] * I[n] * out->R[n+1] elements in the layout above.
 * workspace, workspace_bytes   device scratch of at least
 *        tt_round_workspace_size(x) bytes (256-byte aligned).
 * N = 1 copies the single core.  A zero tensor returns ranks all 1 and zero
 * cores.  Synchronizes `stream` before returning.
 *
 * Host memory: the cores of x and of out may also be page-locked host memory
 * mapped into the device's address space (cudaHostAlloc, or cudaHostRegister
 * with unified addressing), as well as memory of the current device or managed
 * memory.  The kernels then read each input core once and write each output core
 * once over the host link, with no staging copy: the orthogonalization sweep
 * reads every core exactly once and the arithmetic (not the link) bounds it.
 * Any other pointer (unregistered host memory, another device's memory) returns
 * TT_ERR_INVALID_ARG before anything is queued.
 */
int tt_round(const tt_tensor *x, double eps, int precision, tt_tensor *out, void *workspace, size_t workspace_bytes,
             void *stream);

/*
 * Orderings of TT rounding (Sec. 3.4; the RLR and LRL variants of Sec. 4.3.2).
 * TT_ORDER_RLR: right-to-left orthonormalization, then truncation from the left
 * (Alg. 2, Alg. 6; what tt_round computes).  TT_ORDER_LRL: left-to-right
 * orthonormalization (QR of every V(X_n), n = 1..N-1, R pushed into core n+1),
 * ||X|| = ||X_N||_F, then truncation from the right: for n = N..2 the SVD of
 * H(X_n) (through the QR of H(X_n)^T), the same rank rule with delta =
 * eps ||X|| / sqrt(N-1), H(Y_n) <- the leading L_{n-1} right singular vectors
 * (rows orthonormal) and V(X_{n-1}) <- V(X_{n-1}) V_hat Sigma_hat.  Both satisfy
 * ||X - Y|| <= eps ||X||; their results differ by O(delta).
 */
typedef enum { TT_ORDER_RLR = 0, TT_ORDER_LRL = 1 } tt_order;

/* Workspace bytes of tt_round_ordered (TT_ORDER_LRL: about twice the input size
 * more than tt_round, for the mode-reversed copies described below). */
int tt_round_ordered_workspace_size(const tt_tensor *x, int precision, int order, size_t *bytes);

/*
 * tt_round in the given ordering; arguments, results and errors as tt_round
 * (TT_ORDER_RLR is tt_round itself).  TT_ORDER_LRL runs the right-to-left
 * kernels on the mode-reversed tensor (core m = X_{N-1-m} with its rank indices
 * swapped, whose transposed horizontal unfoldings are the vertical unfoldings
 * of X up to a row permutation, which leaves every R factor unchanged), then
 * reverses the result: two extra memory-bound passes, one over the input and one
 * over the output, in the workspace.  Synchronizes `stream`.
 */
int tt_round_ordered(const tt_tensor *x, double eps, int precision, int order, tt_tensor *out, void *workspace,
                     size_t workspace_bytes, void *stream);

/* Workspace bytes of tt_round_hadamard (those of rounding the product's shape). */
int tt_round_hadamard_workspace_size(const tt_tensor *a, const tt_tensor *b, int precision, size_t *bytes);

/*
 * Rounding of a Hadamard product (Sec. 3.2.2 followed by Alg. 2 / Alg. 6) without
 * forming it: Y = round(A o B, eps) with the same result as tt_hadamard followed by
 * tt_round, but the product's cores (R_A R_B x I x R_A' R_B', Kronecker order as in
 * tt_hadamard) are never written: the kernels that read input cores (the
 * orthogonalization sweep and the first core) form each entry A_n(p, i, s) B_n(q, i, t)
 * where they use it.  In FP32 storage the products are formed exactly (a double-float
 * pair for TT_PREC_FP32X2), not rounded to FP32 first.  a and b share N, dtype and I;
 * the product ranks must be supported (as tt_round's); out->cores[n] must hold
 * R_A[n] R_B[n] I[n] R_A[n+1] R_B[n+1] elements; out->R receives the new ranks.
 * Workspace and errors as tt_round.  Synchronizes `stream`.
 */
int tt_round_hadamard(const tt_tensor *a, const tt_tensor *b, double eps, int precision, tt_tensor *out,
                      void *workspace, size_t workspace_bytes, void *stream);

/*
 * Sharded rounding: one tensor distributed over `world_size` shards (processes,
 * one per GPU), each owning a contiguous range of the slices of every core -- the
 * 1 x P x 1 distribution of Sec. 3.1 (Fig. 2): core n of shard p holds slices
 * [begin_p, end_p) of mode n, begin_p = floor(p I_n / world_size) (tt_shard_range),
 * as an R_{n-1} x (end_p - begin_p) x R_n core in the layout above.
 *
 * Every tall-skinny QR of Alg. 6 then spans the shards (Sec. 3.3): each shard
 * factors its row block with the single-GPU kernels, the shards all-gather their
 * b x b triangular factors, and every shard factors the same tree over the
 * gathered factors (the redundant root of the butterfly TSQR, Alg. 3, for any
 * number of shards).  Applying Q (Alg. 4) then needs no communication: each shard
 * applies the shard-level tree and keeps its own block.  A rounding exchanges one
 * payload per tall-skinny QR (2(N-1) of them) plus one before any work (the
 * arguments of all shards must agree) and one at the end (so that every shard
 * returns the same status): 2N all-gathers per call, in the same order on every
 * shard, whatever fails.  The first payload is a 16-byte header; the others are
 * 16 + 8 b_max^2 bytes, b_max the largest input rank.
 */
typedef int (*tt_allgather_fn)(const void *send, void *recv, size_t bytes, void *ctx);

typedef struct {
  int32_t rank;             /* this shard, 0 <= rank < world_size */
  int32_t world_size;       /* number of shards, 1..1024 */
  const int64_t *I_global;  /* host array [N]: mode sizes of the whole tensor, each
                               >= world_size; x->I[n] must be the length of this
                               shard's range of mode n */
  tt_allgather_fn allgather;/* gathers `bytes` from every shard's `send` (host memory)
                               into `recv` (world_size * bytes, shard p's at offset
                               p * bytes) on every shard; returns 0 on success.  Called
                               from the thread that called tt_round_sharded */
  void *ctx;                /* passed to allgather */
} tt_shard;

/* Range [*begin, *end) of the slices of a mode of size I that shard `rank` of
 * `world_size` owns.  Host only; TT_ERR_INVALID_ARG unless 1 <= world_size <= I,
 * world_size <= 1024 and 0 <= rank < world_size. */
int tt_shard_range(int64_t I, int32_t world_size, int32_t rank, int64_t *begin, int64_t *end);

/* Workspace bytes of tt_round_sharded on this shard (x is the local tensor). */
int tt_round_sharded_workspace_size(const tt_tensor *x, int precision, const tt_shard *shard, size_t *bytes);

/*
 * TT rounding (Alg. 2 / Alg. 6, RLR ordering) of the tensor whose shard `rank`
 * is x.  Every shard calls this with the same eps, precision, I_global, ranks and
 * dtype; on return out (as in tt_round, local mode sizes) holds this shard's
 * slices of the rounded cores and out->R the new ranks, the same on every shard.
 * The result equals tt_round's on the whole tensor up to rounding errors (the
 * reduction tree differs).  A shard whose own arguments are wrong (x->I not its
 * range, workspace short, cores not device-accessible) still takes part in the
 * first all-gather and every shard returns the first such error in rank order;
 * arguments that disagree between shards return TT_ERR_INVALID_ARG on all; a
 * failed allgather call returns TT_ERR_COMM (after the first all-gather, the
 * remaining all-gathers of the call are still made, so that the shards stay in
 * step).  A NULL shard, a NULL callback or a rank outside [0, world_size) returns
 * TT_ERR_INVALID_ARG without calling allgather.  world_size 1 is tt_round.
 * Synchronizes `stream` at every all-gather.
 */
int tt_round_sharded(const tt_tensor *x, double eps, int precision, const tt_shard *shard, tt_tensor *out,
                     void *workspace, size_t workspace_bytes, void *stream);

/*
 * Orthonormalization with explicit factors (Alg. 1, parallel form Alg. 5; the
 * left-hand side is its mirror, Sec. 3.4).  TT_ORTH_RIGHT: for n = N..2 the QR of
 * H(X_n)^T = Q R, H(Y_n) <- Q^T (orthonormal rows), R pushed into core n-1; core 1
 * carries the tensor's scale, ||X|| = ||Y_1||_F.  TT_ORTH_LEFT: for n = 1..N-1 the
 * QR of V(X_n) = Q R, V(Y_n) <- Q (orthonormal columns), R pushed into core n+1;
 * ||X|| = ||Y_N||_F.  Ranks become K (right: K_n = min(R_n, I_n K_{n+1}); left:
 * the mirror), known from the shapes.
 */
typedef enum { TT_ORTH_RIGHT = 0, TT_ORTH_LEFT = 1 } tt_orth_side;

/* Workspace bytes of tt_orthonormalize (TT_ORTH_LEFT adds the mode-reversed copies). */
int tt_orthonormalize_workspace_size(const tt_tensor *x, int precision, int side, size_t *bytes);

/*
 * x, precision, out and workspace as in tt_round: out->cores[n] must hold
 * x->R[n] I[n] x->R[n+1] elements; out->R is written (on the host, before any
 * work runs).  The input tensor's scale is carried by the end core (first core
 * for TT_ORTH_RIGHT, last for TT_ORTH_LEFT); in FP32 storage a tensor whose norm
 * is outside the FP32 range over- or underflows there.  Asynchronous: the work is
 * queued on `stream` and the call returns without synchronizing.
 */
int tt_orthonormalize(const tt_tensor *x, int precision, int side, tt_tensor *out, void *workspace,
                      size_t workspace_bytes, void *stream);

/*
 * Batched rounding of `count` independent tensors (each as in tt_round, eps[k]
 * per tensor, one precision for all).  The batch is spread over up to
 * TT_BATCH_SLOTS internal CUDA streams forked from `stream` and joined back
 * into it, each slot owning one region of the workspace.  Tensors are assigned
 * largest first (work ~ sum_n R_{n-1} I_n R_n max(R_{n-1}, R_n)), each to the
 * slot with the least work so far; ties go to the lowest slot.  The library
 * creates those streams and their events once per device on first use and
 * keeps them until exit.  Members are planned in the batch context of the
 * tile table (see tt_autotune_batched).
 */
#define TT_BATCH_SLOTS 16

/* Workspace bytes for a batch (slots plus device space for ranks and status). */
int tt_round_batched_workspace_size(int32_t count, const tt_tensor *xs, int precision, size_t *bytes);

/* Synchronous: fills outs[k].R; returns the first non-OK status of the batch. */
int tt_round_batched(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                     void *workspace, size_t workspace_bytes, void *stream);

/*
 * Asynchronous form of tt_round_batched: queues everything on `stream` (and the
 * slot streams joined into it) and returns without synchronizing, so the call
 * can be captured into a CUDA graph.  Ranks of tensor k go to the device array
 * ranks_dev at offset sum_{j<k} (xs[j].N + 1), its status word to
 * status_dev[k] (both caller-owned device int32 arrays); outs[k].R is not
 * written.  Shapes, pointers and eps are read at call time.
 */
int tt_round_batched_async(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                           int32_t *ranks_dev, int32_t *status_dev, void *workspace, size_t workspace_bytes,
                           void *stream);

/*
 * Tile autotuning.  Each core of a rounding is split into P leaves (CTAs) over
 * its I_n slices (the leaves of the TSQR tree, Sec. 4.1), each leaf walking its
 * slab in tiles of Tt slices.  Without tuning the library takes P = 2 leaves per
 * SM while each leaf gets at least 16 b rows of the core's tall-skinny matrix, else
 * one leaf per SM, at most I_n, and for a batch member at most one leaf per two SMs;
 * with two leaves per SM (and for batch members) the largest tile that lets two
 * leaves share an SM, with one leaf per SM the largest tile that fits.  The
 * tuner times complete roundings of the given tensor(s) on the GPU and records,
 * per core class (precision, context, I_n, R_{n-1}, R_n and the ranks after the
 * orthogonalization sweep), the fastest (P, Tt) it tried, in a table that every
 * later plan of the process consults (including tt_norm's, which shares the
 * orthogonalization sweep).  A tuned plan computes the same rounding with a
 * different reduction tree, so results agree with the untuned ones to rounding
 * error, not bit for bit; ranks are chosen identically unless a singular value
 * sits within rounding error of the threshold.
 *
 * Workspace sizes depend on the table: query them after tuning (or importing),
 * and re-query whenever tt_tune_generation() has changed.  A call given a
 * workspace sized under an older table returns TT_ERR_WORKSPACE.
 */

/* Workspace covering every candidate plan of tt_autotune for x. */
int tt_autotune_workspace_size(const tt_tensor *x, int precision, size_t *bytes);

/*
 * Tunes the core classes of x for a single rounding: coordinate descent over
 * the classes, largest first, over P in {P_default, SMs/2, SMs, 2 SMs, 3 SMs,
 * 4 SMs} (clamped to [1, min(I_n, 1024)]) and Tt in {T_default, T_default/2,
 * largest that fits}; each candidate is timed (best of two) by complete
 * roundings of x into out, and kept if it is 2 % faster than the incumbent.
 * On return `out` holds a valid rounding of x (as from tt_round) and the table
 * holds the winners.  Same argument rules and errors as tt_round, plus
 * TT_ERR_WORKSPACE below tt_autotune_workspace_size.  Synchronizes `stream`.
 */
int tt_autotune(const tt_tensor *x, double eps, int precision, tt_tensor *out, void *workspace,
                size_t workspace_bytes, void *stream);

/* Workspace covering every candidate policy of tt_autotune_batched. */
int tt_autotune_batched_workspace_size(int32_t count, const tt_tensor *xs, int precision, size_t *bytes);

/*
 * Tunes a batch: one policy for all members, P = min(c SMs, I_n) with c in
 * {4, 2, 1, 1/2, 1/4, 1/8, 1/16} and Tt either T_default or the largest that
 * fits.  Each leaf cap is timed with T_default by one complete batched rounding
 * into outs (after one untimed rounding with the current plans), then the other
 * tile rule at the best cap (kept if 2 % faster); the winner is recorded for
 * every member class in the batch context.  Arguments and errors as
 * tt_round_batched.
 */
int tt_autotune_batched(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                        void *workspace, size_t workspace_bytes, void *stream);

/*
 * The table as text, one entry per line "prec ctx I R0 R1 K0 K1 P Tt" (ctx 0 =
 * single rounding, 1 = batch member; P or Tt 0 = default) after one comment
 * line.  *length = bytes needed including the terminating NUL; buf may be NULL
 * to query it; TT_ERR_WORKSPACE if capacity is short.
 */
int tt_tune_export(char *buf, size_t capacity, size_t *length);

/* Adds the entries of a text in tt_tune_export's format (lines starting with '#'
 * and blank lines ignored).  TT_ERR_INVALID_ARG, with the table unchanged, if any
 * line is malformed or out of range (prec 1..3, ctx 0..1, I >= 1, 1 <= K0 <= R0
 * <= TT_MAX_RANK, 1 <= K1 <= R1 <= TT_MAX_RANK, 0 <= P <= 1024, Tt >= 0). */
int tt_tune_import(const char *text);

/* Empties the table (plans go back to the defaults). */
int tt_tune_clear(void);

/* Counter bumped by every change of the table. */
uint64_t tt_tune_generation(void);

/*
 * Summation (Sec. 3.2.1): Z = A + B.  Interior slices are block diagonal
 * diag(A_n(i), B_n(i)); the first core is [A_1 B_1], the last [A_N; B_N]; the
 * ranks add (N = 1: the entrywise sum).  out->R is written by the routine;
 * out->cores[n] must hold (Ra[n]+Rb[n]) I[n] (Ra[n+1]+Rb[n+1]) elements (with
 * the end ranks 1).  Asynchronous.
 */
int tt_add(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, void *stream);

/*
 * Hadamard product (Sec. 3.2.2): Z_n(i) = A_n(i) kron B_n(i); ranks multiply.
 * Kronecker order: row (p, q) of the slice is p * Rb + q.  out->R is written by
 * the routine; out->cores[n] must hold Ra[n]Rb[n] I[n] Ra[n+1]Rb[n+1] elements.
 * Asynchronous.
 */
int tt_hadamard(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, void *stream);

/* Workspace bytes tt_dot needs for inputs a, b. */
int tt_dot_workspace_size(const tt_tensor *a, const tt_tensor *b, size_t *bytes);

/*
 * Inner product <A, B> (Sec. 3.2.3): W_0 = 1, H(Z_n) = W_{n-1} H(A_n),
 * W_n = V(B_n)^T V(Z_n), result = W_N.  Partial sums over slices are reduced
 * in a fixed order in FP64.  Writes the host double *result; synchronizes.
 */
int tt_dot(const tt_tensor *a, const tt_tensor *b, double *result, void *workspace, size_t workspace_bytes,
           void *stream);

/*
 * Size of the fixed device scratch array behind tt_dot_noalloc (8 MiB).
 */
#define TT_DOT_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)

/*
 * tt_dot without any memory allocation, for callers that cannot allocate
 * device memory: code whose host framework owns every device allocation (a
 * fixed pool or arena it does not expose), loops where the device-wide
 * synchronization of cudaMalloc/cudaFree is not acceptable, or embedded and
 * plugin contexts where allocating is forbidden.  The paper has no counterpart:
 * this is the same inner product as tt_dot (same kernels, same result) with its
 * scratch taken from a fixed array of TT_DOT_NOALLOC_SCRATCH_BYTES that lives in
 * device memory of every GPU that loads this library, until the process exits.
 *
 * a, b, result and stream as in tt_dot; no workspace argument.  Neither this
 * routine nor anything it calls allocates (no cudaMalloc, cudaFree or
 * allocating library call).  Returns TT_ERR_UNSUPPORTED, having queued nothing,
 * when the scratch tt_dot would need (tt_dot_workspace_size(a, b), about
 * 8 (2 max_n Ra[n]Rb[n] + max_n min(I[n], 304) Ra[n+1]Rb[n+1]) bytes) exceeds
 * TT_DOT_NOALLOC_SCRATCH_BYTES; two tensors whose ranks are all r fit for
 * r <= 58.
 * The first call on a device looks up that device's scratch address, with the
 * device current; make that first call before any stream capture.  The address
 * is kept for the life of the process: after cudaDeviceReset (or anything else
 * that destroys the device's primary context) it is stale, so do not call this
 * routine on that device again in the same process.  All calls
 * share the one array and it keeps the last call's contents (every value a call
 * reads it writes first): calls whose work overlaps on the GPU -- other streams,
 * other host threads -- race and give wrong results.  Synchronizes `stream`.
 */
int tt_dot_noalloc(const tt_tensor *a, const tt_tensor *b, double *result, void *stream);

/* Workspace bytes tt_norm needs for input x. */
int tt_norm_workspace_size(const tt_tensor *x, size_t *bytes);

/*
 * Norm through orthonormalization (Sec. 3.2.4, second approach): the
 * right-to-left sweep of tt_round, then ||X|| = Frobenius norm of the first
 * core.  Free of the cancellation of sqrt(<X, X>).  Writes the host double
 * *result; synchronizes.
 */
int tt_norm(const tt_tensor *x, double *result, void *workspace, size_t workspace_bytes, void *stream);

/* Static description of a status code. */
const char *tt_status_string(int status);

/*
 * Diagnostics (no counterpart in the paper): per kernel class, the number of
 * kernels this library launched and, while tracing is on, their device time.
 */
typedef enum {
  TT_K_S1_LEAF = 0,     /* right-to-left sweep: slab push + Householder QR (Alg. 6, first loop) */
  TT_K_TREE_FACTOR = 1, /* reduction tree of triangular factors (TSQR, Alg. 3) */
  TT_K_TREE_APPLY = 2,  /* root-to-leaf application of stored tree reflectors (Alg. 4) */
  TT_K_S2_LEAF = 3,     /* left-to-right sweep: apply stored Q_n, QR of V(Y_n) slabs */
  TT_K_S2_OUT = 4,      /* left-to-right sweep: output core Q' U_hat */
  TT_K_SVD = 5,         /* FP64 Jacobi SVD of the root factor and rank choice */
  TT_K_ADD = 6,
  TT_K_HADAMARD = 7,
  TT_K_DOT = 8,
  TT_K_MISC = 9,        /* control-block set-up, norm reductions */
  TT_K_COUNT = 10
} tt_kernel_kind;

/*
 * enable != 0: reset all counters and start bracketing every launch with two
 * CUDA events recorded on the launch's own stream; enable == 0: stop recording
 * events (counters keep counting).  Not thread-safe with concurrent calls.
 */
int tt_trace(int enable);

/*
 * For kernel class `kind`: *launches = kernels launched since the last
 * tt_trace(1); *milliseconds = summed device time of the launches recorded
 * while tracing was on (waits for those events).  Either pointer may be NULL.
 */
int tt_trace_read(int kind, int64_t *launches, double *milliseconds);

#ifdef __cplusplus
}
#endif

#endif /* TTGB_TT_H */
