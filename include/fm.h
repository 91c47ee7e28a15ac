/*
 * fm.h -- C ABI of the GB300 structured-operator library (libfastmat_gb300.so).
 *
 * The library applies composed structured linear operators to blocks of
 * columns on one GPU: the forward transform phi_A(X) = A X (Eq. (3) of the
 * fastmat paper, arXiv 1710.09578) and the backward transform
 * beta_A(Y) = A^H Y (Eq. (4)), plus a batched FISTA solver for the
 * l1-regularised least-squares problem of Eq. (8) built on those two calls.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Column blocks.  A block of K columns of length n is stored column by column:
 *   column k starts at element k*ld of the buffer, its n elements are
 *   contiguous, ld >= n.  (A C-contiguous torch tensor of shape [K, n] is such a
 *   block with ld = n.)  Element types are given by fm_dtype; complex types are
 *   interleaved (re, im).
 * Pointers.  Constructor parameter arrays may be host or device pointers (they
 *   are copied with cudaMemcpyDefault and may be freed or changed afterwards:
 *   operators are immutable, Sec. 2.1.1 of the paper).  Data buffers passed to
 *   fm_forward / fm_backward / fm_fista are DEVICE pointers owned by the
 *   caller.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  All device work is enqueued on it; no call synchronises the
 *   device unless stated.  Transform kernels are launched with programmatic
 *   dependent launch: they may become resident while the previous kernel of the
 *   stream finishes, but touch memory only after it has completed, so stream
 *   order is kept as usual (also inside captured CUDA graphs).
 * Errors.  Every call returns fm_status.  Argument checks run before any
 *   launch and leave outputs untouched.  Asynchronous CUDA failures surface as
 *   FM_ERR_CUDA from a later call.  fm_last_error() gives a one-line message
 *   for the calling thread.  Nothing throws across this ABI.
 * Ownership.  Constructors return a handle with one reference.  Composites
 *   hold a reference to each child, so children may be released right after
 *   the composite is built.  fm_release drops one reference.
 */
#ifndef FM_H
#define FM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fm_op_s* fm_op;
typedef struct fm_batch_s* fm_batch;

typedef enum {
  FM_OK = 0,
  FM_ERR_INVALID_ARG = 1, /* null pointer, bad count or flag                        */
  FM_ERR_SHAPE = 2,       /* sizes of composed operators or buffers disagree         */
  FM_ERR_DTYPE = 3,       /* element type not accepted by the operator               */
  FM_ERR_UNSUPPORTED = 4, /* valid request outside what this build implements        */
  FM_ERR_ALIAS = 5,       /* output overlaps input where in-place is not allowed      */
  FM_ERR_OOM = 6,         /* device allocation failed                                */
  FM_ERR_CUDA = 7,        /* CUDA runtime error (launch or earlier asynchronous one) */
  FM_ERR_TIMEOUT = 8,     /* a bounded device wait ran out                           */
  FM_ERR_NUMERIC = 9      /* non-finite value met where a finite one is required     */
} fm_status;

typedef enum { FM_I8 = 0, FM_I32 = 1, FM_F32 = 2, FM_F64 = 3, FM_C64 = 4, FM_C128 = 5 } fm_dtype;

/* Arithmetic of the Hadamard transform (the Sylvester matrix is exact +-1):
 *   FM_HAD_FP32   f32 or c64 data, FP32 adds;
 *   FM_HAD_BF16   f32 data rounded to BF16 and multiplied by 16x16 +-1 tiles on
 *                 the tensor cores with FP32 accumulation (relative error ~1e-3);
 *   FM_HAD_BF16X2 as BF16 but each stage splits x = hi + lo into two BF16
 *                 parts and accumulates both products (FP32-level accuracy);
 *   FM_HAD_INT8   int8 data, int32 output, exact. */
typedef enum { FM_HAD_FP32 = 0, FM_HAD_BF16 = 1, FM_HAD_BF16X2 = 2, FM_HAD_INT8 = 3 } fm_had_mode;

/* ---------------------------------------------------------------- constructors */

/* Fourier matrix of Eq. (1), read 0-based: F[k, j] = exp(-2 pi i j k / n); F^H has
 * the opposite sign and no 1/n.  ortho = 1 scales both by 1/sqrt(n).
 * n must be a power of two, 1 <= n <= 2^24 (FM_ERR_UNSUPPORTED otherwise). */
fm_status fm_fourier(int64_t n, int ortho, fm_op* out);

/* Circulant matrix C[i, j] = c[(i - j) mod n] with first column c (Eq. (5):
 * C x = ifft(fft(c) * fft(x)); Sec. 2.1.1: C = F^H Diag(F c / n) F with the
 * spectrum computed once, in FP64, at construction).  dt in {F32, F64, C64, C128}.
 * n a power of two, 1 <= n <= 2^24. */
fm_status fm_circulant(const void* c, int64_t n, fm_dtype dt, void* stream, fm_op* out);

/* Toeplitz matrix (Sec. 2.1.1: non-circular convolution in the frequency domain),
 * rows x cols, T[i, j] = t[i - j] for i >= j and t[rows - 1 + j - i] for i < j, i.e.
 * t = [first column (rows entries); first row without t0 (cols - 1 entries)].
 * Applied through a circulant embedding of length L = 2^ceil(log2(rows + cols - 1)),
 * L <= 2^24.  dt in {F32, F64, C64, C128}. */
fm_status fm_toeplitz(const void* t, int64_t rows, int64_t cols, fm_dtype dt, void* stream,
                      fm_op* out);

/* Circulant whose first column is a pseudo-random +-1 sequence from a linear feedback shift
 * register (the LFSRCirculant of Sec. 4; the paper gives no register conventions, so:) a
 * Fibonacci register of nbits bits (1..63) starting from a nonzero `state`; each step outputs
 * o = s & 1, forms f = parity(s & taps) and shifts s <- (s >> 1) | (f << (nbits - 1)); the column
 * holds c[k] = +1 for o_k = 0 and -1 for o_k = 1, for the first n outputs (n a power of two,
 * <= 2^24; a maximal-length sequence has period 2^nbits - 1).  The taps of x^m + x^a + 1 are
 * bits 0 and a.  A real circulant, as fm_circulant. */
fm_status fm_lfsr_circulant(int32_t nbits, uint64_t taps, uint64_t state, int64_t n, void* stream, fm_op* out);

/* Sylvester Hadamard matrix H[i, j] = (-1)^popcount(i & j), natural order,
 * unnormalised, n = 2^log2n, 0 <= log2n <= 24 (BF16 modes: 4 <= log2n <= 16).
 * Symmetric, so forward and backward are the same map. */
fm_status fm_hadamard(int log2n, fm_had_mode mode, fm_op* out);

/* Diagonal matrix Diag(d) (Eq. (7)): y_i = d_i x_i, adjoint conj(d_i) y_i.
 * dt in {F32, F64, C64, C128}. */
fm_status fm_diag(const void* d, int64_t n, fm_dtype dt, void* stream, fm_op* out);

/* Row selection P (the operator P of Eq. (7); "random selection of rows" in the
 * compressed model of Sec. 3): m x n, y_r = x_{idx[r]}; the adjoint zero-fills and
 * scatters.  idx (int32, host or device) must hold m distinct values in [0, n);
 * FM_ERR_INVALID_ARG otherwise (checked on the host at construction). */
fm_status fm_partial(const int32_t* idx, int64_t m, int64_t n, void* stream, fm_op* out);

/* Compositions (Sec. 2.1.1: the transforms of a composite are built from the
 * transforms of its terms).  terms/factors/blocks: k >= 1 handles.
 *   product  terms[0] * terms[1] * ... * terms[k-1] (terms[k-1] is applied first);
 *   sum      terms[0] + ... + terms[k-1], all the same shape;
 *   blkdiag  block-diagonal arrangement, x split into consecutive segments;
 *   kron     factors[0] (x) ... (x) factors[k-1] in numpy.kron order (the first
 *            factor acts on the most significant index digit), applied as mode
 *            products;
 *   hermitian  A^H as an operator (forward of it is the backward of A). */
fm_status fm_product(const fm_op* terms, int k, fm_op* out);
fm_status fm_sum(const fm_op* terms, int k, fm_op* out);
fm_status fm_blkdiag(const fm_op* blocks, int k, fm_op* out);
fm_status fm_kron(const fm_op* factors, int k, fm_op* out);
fm_status fm_hermitian(fm_op A, fm_op* out);

/* Block matrix [B_ij] of nrows x ncols operators (the block arrangement of the ultrasound model
 * H = [H_ij] of Sec. 3): blocks[i * ncols + j] is block (i, j); the blocks of one block row share
 * their row count and those of one block column their column count (FM_ERR_SHAPE otherwise).
 * Forward: output segment i = sum_j B_ij (input segment j); backward: segment j = sum_i
 * B_ij^H (segment i).  Holds a reference to every block. */
fm_status fm_blocks(const fm_op* blocks, int nrows, int ncols, fm_op* out);

/* Two-level Toeplitz matrix (a 2-D non-cyclic convolution, the blocks H_ij of Sec. 3) of shape
 * (r1 r2) x (c1 c2), vectors read as row-major r1 x r2 (output) and c1 x c2 (input) grids:
 *   T2[(i1, i2), (j1, j2)] = t[k(i1, j1; r1) * (r2 + c2 - 1) + k(i2, j2; r2)],
 *   k(i, j; r) = i - j for i >= j and r - 1 + j - i for i < j (the 1-D rule of fm_toeplitz on
 *   each level), so t is a row-major (r1 + c1 - 1) x (r2 + c2 - 1) array (host or device).
 * Built as Eq. (7) writes it: the zero-padding of the input to the L1 x L2 grid
 * (L = 2^ceil(log2(r + c - 1)) per level), (F_L1 (x) F_L2)^H Diag(h) (F_L1 (x) F_L2) with
 * h = (F_L1 (x) F_L2) e / (L1 L2) computed in FP64 from the embedded generator e, and the
 * truncation to the r1 x r2 block: the handle returned is that Product.  It is complex (its
 * output for a real generator and real input is real up to rounding: request the real type
 * to keep the real part).  L1 L2 <= 2^24. */
fm_status fm_toeplitz2(const void* t, int64_t r1, int64_t c1, int64_t r2, int64_t c2, fm_dtype dt, void* stream,
                       fm_op* out);

/* ---------------------------------------------------------------- queries */

fm_status fm_shape(fm_op A, int64_t* rows, int64_t* cols);
/* 1 if every entry of A is real (real operators keep real data real). */
fm_status fm_is_real(fm_op A, int* is_real);
/* Element type of phi_A / beta_A output for input type `in`:
 * complex if A or the input is complex; int8 -> int32 for FM_HAD_INT8 Hadamard;
 * otherwise the input type.  FM_ERR_DTYPE if A does not accept `in`. */
fm_status fm_out_dtype(fm_op A, fm_dtype in, fm_dtype* out);

/* ---------------------------------------------------------------- transforms */

/* Y = A X (forward, Eq. (3)) for ncols columns.  X: cols(A) x ncols block of type
 * xdt with leading dimension ldx; Y: rows(A) x ncols block of type ydt with leading
 * dimension ldy.  ydt is fm_out_dtype(A, xdt), or, where that type is complex, the real
 * type of the same precision (F32 for C64, F64 for C128): then Y = Re(A X).  The real
 * part is what a real-valued parameterisation needs: for real x the map x -> A x into
 * C^m, seen as R^2m, has the adjoint y -> Re(A^H y), so the gradient of a loss with
 * respect to a real x is fm_backward with a real output type.  Y must not overlap X.
 * Intermediate buffers come from a per-operator workspace that grows on demand
 * (call fm_reserve first to keep the call free of allocation, e.g. before
 * capturing it in a CUDA graph). */
fm_status fm_forward(fm_op A, const void* X, int64_t ldx, fm_dtype xdt, void* Y, int64_t ldy,
                     fm_dtype ydt, int64_t ncols, void* stream);

/* X = A^H Y (backward, Eq. (4)); shapes and rules mirror fm_forward. */
fm_status fm_backward(fm_op A, const void* Y, int64_t ldy, fm_dtype ydt, void* X, int64_t ldx,
                      fm_dtype xdt, int64_t ncols, void* stream);

/* Grow A's workspace for up to ncols columns of type xdt (both directions). */
fm_status fm_reserve(fm_op A, int64_t ncols, fm_dtype xdt, void* stream);

/* Circulant transform that allocates no device memory.  (The paper has no counterpart:
 * this is a deployment aid, not part of the method.)
 * For callers that cannot allocate device memory while they apply an operator -- a
 * program whose device memory belongs to another allocator or to a fixed budget, or code
 * that must avoid the implicit device synchronisation of cudaMalloc / cudaFree.  It
 * computes the same result as fm_forward (adjoint = 0) or fm_backward (adjoint = 1) of
 * the Circulant operator C on ncols complex64 columns (X, Y: device buffers, leading
 * dimensions ldx, ldy >= n; Y must not overlap X), but the scratch of the two-pass plan
 * used for n > 16384 comes from a fixed 16 MiB array in the library's device image instead
 * of the operator's growable workspace.  That array is reserved on a device when the first
 * Circulant operator is built there (fm_circulant looks up its device address, which loads
 * it) and held until the process exits.  The call itself calls no cudaMalloc, cudaFree or
 * allocating routine and reads the address fm_circulant stored.
 * Limits and rules:
 *   - the scratch needed is n * ncols * 8 bytes when n > 16384 (nothing below that); a
 *     call needing more than 16 MiB returns FM_ERR_UNSUPPORTED: split the columns (n = 2^18
 *     takes up to 8 columns per call);
 *   - C must come from fm_circulant on the current device (FM_ERR_INVALID_ARG otherwise);
 *   - after cudaDeviceReset every operator of that device is invalid, and so is the stored
 *     address: build a new Circulant operator there (which stores it again) before calling;
 *   - all calls share the one array, which keeps what the last call wrote (every element
 *     a call reads it has written first, so nothing needs clearing): calls that overlap
 *     on the GPU -- on different streams, or from different threads -- race, so serialise
 *     them (one stream). */
fm_status fm_circulant_apply_noalloc(fm_op C, int adjoint, const void* X, int64_t ldx, void* Y, int64_t ldy,
                                     int64_t ncols, void* stream);

/* Gradient with respect to the parameter vector of `leaf` (Sec. 2.1.1: operators built from
 * parameter vectors), for a real loss of Y = A X with upstream gradient G = dloss/dconj(Y) (the
 * convention of fm_backward: the gradient of X is A^H G).  leaf is a Diag (parameter d, n
 * entries), Circulant (first column c, n entries) or Toeplitz (generator t = [first column;
 * first row without t0], rows + cols - 1 entries) operator that is A itself or appears once,
 * not as an adjoint, among the terms of A's (nested) product.  Y is bilinear in (theta, X), so
 *   grad[k] = sum over columns and over the entries (i, j) of the leaf holding theta_k of
 *             G_leaf[i] conj(Z[j]),
 * the real part for a real leaf, where Z is the leaf's input (the terms applied before it,
 * recomputed from X; nothing of the forward pass is stored) and G_leaf the gradient at its
 * output (the adjoints of the terms applied after it, applied to G).  For a circulant or
 * Toeplitz leaf the sum is the circular correlation (1/L) F^H sum_c (F G_leaf) conj(F Z) of the
 * columns zero-padded to the leaf's transform length L.
 * X: cols(A) x ncols (dtype xdt in F32, F64, C64, C128, leading dimension ldx), G: rows(A) x
 * ncols of dtype fm_out_dtype(A, xdt) (ldg), grad: device vector of the parameter length, of
 * dtype complex_of(xdt) for a complex leaf and the real type of xdt's precision for a real
 * one; it is overwritten.  Intermediates come from A's workspace (grown on demand). */
fm_status fm_param_grad(fm_op A, fm_op leaf, const void* X, int64_t ldx, fm_dtype xdt, const void* G, int64_t ldg,
                        fm_dtype gdt, int64_t ncols, void* grad, fm_dtype grad_dt, void* stream);

/* Orthogonal matching pursuit (cited in Sec. 3 beside (F)ISTA; Sec. 4 names its rank-1 update
 * form) for one right-hand side b (rows(A) entries) with K steps:
 *   r_0 = b, S = [];  for k = 1..K: c = A^H r_{k-1}, j = argmax_i |c_i| (the lowest index among
 *   equal magnitudes), S += [j], x_S = argmin ||A_S z - b||, r_k = b - A_S x_S;  x[S] = x_S.
 * A enters only through fm_backward (correlations) and fm_forward (the column A e_j); the least
 * squares solution is kept as a thin QR factorisation A_S = Q R extended by one column per step
 * (classical Gram-Schmidt applied twice).  dt: C64 or C128 (any operator), or F32 / F64 for a
 * real operator (solved in complex, real part returned).  b, x (cols(A) entries, overwritten)
 * and support (K int32 picks in order, may be NULL) are DEVICE buffers.  1 <= K <= min(rows,
 * cols, 4096).  Reductions run in a fixed order (bit-reproducible).  The call allocates its
 * workspace (Q: K x rows) and synchronises `stream` before it returns. */
fm_status fm_omp(fm_op A, const void* b, fm_dtype dt, int32_t K, void* x, int32_t* support, void* stream);

/* ---------------------------------------------------------------- calibration */

/* Calibration of the execution plan: the GPU form of the paper's calibration step
 * (Sec. 2.1.3), which times an operator's transforms and keeps what it learns.  The settings
 * it chooses, among variants compiled into the library:
 *   kind 0  the split L = N1 x N2 of a transform longer than one tile (Fourier, Circulant or
 *           Toeplitz embedding of length L > 8192), N1 = 2^e with N1, N2 in [2^5, 2^13];
 *   kind 1  the tile shape of an FFT leaf's strided views: 0 automatic (for inner strides >= 16
 *           radix-32 tiles at length 2^10 in FP32, wide tiles of 8 or 16 vectors elsewhere), 1
 *           the default tile (2^12 elements), 2 the wide tile wherever it applies (lengths 2^9
 *           .. 2^10 in FP32, 2^9 in FP64), 3 the wide FP32 tile split into 4 groups of warps that
 *           transform their own vectors with barriers of their own, 4 radix-32 tiles (FP32
 *           lengths 2^9 and 2^10, strided or not: 2^13 elements, 256 threads of 32 elements, so
 *           a transform takes two radix passes instead of three);
 *   kind 2  the radix schedule of an FFT leaf's tiles: 0 the per-length table (radix 16
 *           first), 3 radices of at most 8 (compiled for FP32 tiles of 2^9 .. 2^12);
 *   kind 3  the fused pass of a Kron(Hadamard, ..., Fourier) operator on complex64 columns (L =
 *           the Kron's length): 0 one CTA per [2^a][2^b] tile; 1 each tile on a cluster of two
 *           CTAs that combine the last Hadamard digit through distributed shared memory; 2 a
 *           cluster of four CTAs and the last two digits (tiles of at least 2^11 elements; a
 *           smaller tile takes the pair); 3 the pair, each CTA also prefetching into L2 its rows
 *           of the tile half a residency wave later (the SM count / 2 tiles on);
 *   kind 5  (set only; the calibration does not time it) an FP32 or int8 Hadamard leaf of length
 *           2^15 or 2^16 on plain column blocks (L = the leaf's n): 0 each CTA prefetches into
 *           L2 its block of the column one residency wave later (the default), 1 no prefetch.
 * fm_calibrate times A's forward + adjoint (one warm-up, mean of three) on ncols probe columns
 * of complex_of(dt) for every candidate of every setting of every transform in A, one setting
 * at a time (splits first, then per leaf the tile shape, then the radix schedule), and keeps
 * the fastest in A.  Results are unchanged up to FP rounding.  It allocates and frees its probe
 * buffers and synchronises `stream`; A must not be in use on another stream meanwhile.
 * report (host, optional): one entry per tuned setting, at most max_entries; *n_entries
 * (optional) receives the number of tuned settings (0 for an operator without FFT leaves). */
typedef struct {
  int64_t L;            /* transform length */
  int64_t n1;           /* chosen value (kind 0: N1, N2 = L / N1; 1: tile shape; 2: radix cap; 3: Kron pass) */
  int32_t ncand;        /* candidates timed (<= 8) */
  int64_t cand_n1[8];   /* their values */
  float ms[8];          /* forward + adjoint of A with that value, milliseconds */
  int32_t kind;         /* 0 split, 1 tile shape, 2 radix schedule, 3 fused Kron pass */
} fm_tune_entry;
fm_status fm_calibrate(fm_op A, int64_t ncols, fm_dtype dt, void* stream, fm_tune_entry* report,
                       int32_t max_entries, int32_t* n_entries);
/* Set N1 of every two-pass transform of length L in A (n1 = 0: the default 2^floor(log2(L)/2)),
 * e.g. to restore a calibration result.  FM_ERR_INVALID_ARG if n1 is not a power of two with
 * N1, L / N1 in [2^5, 2^13]; FM_OK if A has no transform of length L.  Same rules about
 * concurrent use as fm_calibrate. */
fm_status fm_set_split(fm_op A, int64_t L, int64_t n1, void* stream);
/* Set one plan setting (kind and value as in fm_tune_entry) of every FFT leaf (kinds 1, 2), fused
 * Kron operator (kind 3) or long Hadamard leaf (kind 5) of length L in A,
 * e.g. to restore a cached calibration.  FM_ERR_INVALID_ARG for a value outside the kind's
 * range; FM_OK if A has no leaf of length L. */
fm_status fm_set_plan(fm_op A, int64_t L, int32_t kind, int64_t value, void* stream);
/* A text description of A's tree (kinds, shapes, real or complex, Hadamard mode, Fourier
 * scaling), for keying cached calibrations; FM_ERR_SHAPE if it needs more than len bytes. */
fm_status fm_signature(fm_op A, char* buf, int32_t len);

/* Dense execution of a small operator (Sec. 2.1.3: below some size a plain matrix-vector product
 * beats the fast transform).  fm_set_dense(A, 1) materialises A's matrix once (the forward
 * transform of the unit vectors, in FP64 and FP32) and from then on applies A to complex
 * columns of plain blocks as y = M x (M^H y for the backward) from shared memory; real data and
 * strided views keep the fast path, and A inside a Product is not fused with its neighbours.
 * A: a Fourier, Circulant, Toeplitz or FP32 Hadamard operator with rows * cols <= 4096
 * (FM_ERR_UNSUPPORTED otherwise).  fm_set_dense(A, 0) returns to the fast transform.
 * fm_calibrate_dense times A's forward + adjoint on ncols probe columns of dt (C64 or C128)
 * both ways (20 repetitions each, after 3 untimed), keeps the faster and reports both times
 * (milliseconds per forward + adjoint) and the choice (1 dense, 0 fast; any output may be NULL).
 * Both calls allocate and synchronise `stream`; A must not be in use on another stream. */
fm_status fm_set_dense(fm_op A, int dense, void* stream);
fm_status fm_calibrate_dense(fm_op A, int64_t ncols, fm_dtype dt, void* stream, float* ms_fast, float* ms_dense,
                             int32_t* chosen);

/* ---------------------------------------------------------------- FISTA */

/* Batched FISTA (accelerated proximal gradient, cited in Sec. 3) for
 *   min_x 1/2 ||A_i x - b_i||^2 + lambda_i ||x||_1      (Eq. (8) with tau = 2 lambda)
 * on many independent real instances.  Per instance:
 *   lambda = lambda_rel * ||A^T b||_inf;
 *   L = min(safety * lam_hat, max_k |c_hat_k|^2), lam_hat = ||A v_P||^2 after P power
 *       iterations v <- A^T A v / ||A^T A v|| from v_0 = ones / sqrt(n) (c_hat: the
 *       spectrum of the circulant embedding of T);
 *   x_0 = 0, y_1 = 0, t_1 = 1; for k = 1..K: g = A^T (A y_k - b),
 *   x_k = soft(y_k - g / L, lambda / L), t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
 *   y_{k+1} = x_k + (t_k - 1) / t_{k+1} (x_k - x_{k-1})    (accel = 0: y_{k+1} = x_k).
 * FP32 state and transforms; FP64 norms, Rayleigh quotient and objective. */
typedef struct {
  int32_t iters;       /* K, FISTA steps (>= 0)                                       */
  int32_t power_iters; /* P, power iterations for lam_hat (>= 1)                     */
  double lambda_rel;   /* lambda = lambda_rel * ||A^T b||_inf                         */
  double safety;       /* L = min(safety * lam_hat, max |c_hat|^2)                   */
  int32_t accel;       /* 1 FISTA momentum, 0 ISTA                                    */
  int32_t mode;        /* 0: one persistent launch over the whole batch;
                          1: the same steps as separate per-instance launches       */
  int32_t warm;        /* 0: cold start x_0 = y_1 = 0, t_1 = 1, lambda and L computed;
                          1: resume a run that has taken k0 steps (fm_fista_batch only):
                          x holds x_k0, y holds y_{k0+1}, rep->L and rep->lambda hold
                          that run's L and lambda (read, not recomputed), and t_{k0+1}
                          is rebuilt from t_1 = 1 by the same recurrence.  K1 steps, then
                          K2 resumed steps, give the bits of K1 + K2 steps.           */
  int32_t k0;          /* warm: steps the resumed run has taken (>= 0)                */
} fm_fista_params;

/* Per-instance results, DEVICE arrays of length `count` (any may be NULL):
 * L, lambda, final objective 1/2||A x - b||^2 + lambda ||x||_1, status (0 ok,
 * FM_ERR_NUMERIC if a non-finite value appeared).  With p->warm = 1, L and lambda are
 * also inputs (the values of the run being resumed). */
typedef struct {
  double* L;
  double* lambda;
  double* objective;
  int32_t* status;
} fm_fista_report;

/* Batched FISTA on `batch` instances given as operators, each A_i =
 * Product(Partial(idx_i, n_i), Toeplitz(t_i)) with real t_i (n_i x n_i, n_i a power of two in
 * [2^8, 2^14]) and m_i selected rows (other shapes: FM_ERR_UNSUPPORTED).  b[i] (m_i floats) and
 * x[i] (n_i floats, 8-byte aligned) are DEVICE pointers held in HOST arrays of `batch` entries.
 * Every instance starts cold (p->warm must be 0).  The call builds the work list (instances
 * sorted and grouped by size), uploads the pointer arrays, solves all instances in one
 * launch (p->mode = 0) or one launch per instance (p->mode = 1), synchronises `stream` and
 * frees what it built: it allocates, so it cannot be captured in a CUDA graph.  For
 * repeated or captured solves, and to resume a run, build the batch once with
 * fm_batch_create and call fm_fista_batch. */
fm_status fm_fista(const fm_op* A, int64_t batch, const float* const* b, float* const* x, const fm_fista_params* p,
                   const fm_fista_report* rep, void* stream);

/* A batch of `count` instances of the form above, kept for repeated solves.  Building the
 * batch uploads a work list (instances sorted by size) and allocates the per-instance
 * state. */
fm_status fm_batch_create(const fm_op* A, int64_t count, void* stream, fm_batch* out);
void fm_batch_release(fm_batch B);
/* Total rows (sum m_i) and columns (sum n_i) of the batch: the lengths of the packed
 * b and x buffers below. */
fm_status fm_batch_sizes(fm_batch B, int64_t* total_rows, int64_t* total_cols);

/* Solve every instance of B.  b: packed float32 measurements (instance i at offset
 * sum_{j<i} m_j), x: packed float32 solutions (offset sum_{j<i} n_j, 8-byte aligned), both
 * device buffers.  y (optional, packed like x, 8-byte aligned; NULL = a buffer of the batch)
 * receives the momentum state y_{K+1} so that the run can be resumed (p->warm = 1 reads it).
 * No allocation and no host synchronisation: capturable in a CUDA graph. */
fm_status fm_fista_batch(fm_batch B, const float* b, float* x, float* y, const fm_fista_params* p,
                         const fm_fista_report* rep, void* stream);

/* The persistent solve's work list as part of the calibration: each CTA takes the next group
 * of equal-size instances, and the order of the groups decides how the last wave fills the
 * GPU.  fm_batch_tune times one cold persistent solve (p->warm = 0, p->mode = 0, after one
 * untimed) with the groups largest first (0, the default) and smallest first (1), keeps the
 * faster for later solves of B, and reports the milliseconds (ms[2], host, may be NULL) and the
 * choice (*chosen, may be NULL).  It writes x and synchronises `stream`. */
fm_status fm_batch_tune(fm_batch B, const float* b, float* x, const fm_fista_params* p, void* stream, float* ms,
                        int32_t* chosen);
/* Set the work-list order (0 largest first, 1 smallest first), e.g. to restore a tuned choice. */
fm_status fm_batch_set_order(fm_batch B, int32_t order);

/* ---------------------------------------------------------------- tracing */

/* Device time of the library's kernels (profiling; the paper has no counterpart).  Between
 * fm_trace_begin and fm_trace_end every kernel the library launches, on any stream and from
 * any thread, is bracketed by two CUDA events recorded on its stream, up to max_launches
 * launches (later launches run untraced).  An event between two kernels ends the early start
 * of programmatic dependent launch, so traced kernels run one after another.  fm_trace_begin
 * creates the events (host resources, no device memory) and fails if tracing is already on.
 * fm_trace_end waits for the traced launches, copies the first max_entries of them (kernel
 * label, milliseconds) in launch order to out (host, may be NULL), sets *n_entries (may be
 * NULL) to the number of launches seen while tracing was on, and frees the events. */
typedef struct {
  char kernel[64]; /* kernel label, e.g. "fft2_kernel<f32,L=2^10,strided,conv>" */
  float ms;        /* device time between the launch's two events */
} fm_trace_entry;
fm_status fm_trace_begin(int32_t max_launches);
fm_status fm_trace_end(fm_trace_entry* out, int32_t max_entries, int32_t* n_entries);

/* ---------------------------------------------------------------- misc */

void fm_release(fm_op A);
const char* fm_status_string(fm_status s);
/* Message of the last failed call on this thread ("" if none). */
const char* fm_last_error(void);
/* Number of kernels this library has launched in the process so far. */
uint64_t fm_launch_count(void);
/* Library version string. */
const char* fm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FM_H */
