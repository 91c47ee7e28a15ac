// Operator-tree execution: phi_A(X) = A X and beta_A(Y) = A^H Y (Eq. (3), Eq. (4)).
//
// Composite operators are evaluated from the transforms of their terms (Sec. 2.1.1 of
// the paper): a Product applies its terms right to left (its adjoint left to right with
// each term's adjoint), a Sum accumulates, a BlkDiag works on consecutive segments and a
// Kron applies each factor along its own axis of the column seen as a row-major tensor
// (mode products).  Inside a Product a Diag and a row selection next to an FFT-based
// operator (Fourier, Circulant, Toeplitz) are fused into that operator's loads and stores:
// the chain P . Diag(d) . C runs as one kernel, and its adjoint C^H . Diag(d)^H . P^H too.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "exec.h"
#include "kron_hf.h"
#include "fft.h"
#include "fwht.h"
#include "pointwise.h"

namespace fm {

static bool is_float_type(fm_dtype d) { return d == FM_F32 || d == FM_F64 || d == FM_C64 || d == FM_C128; }

static fm_dtype promote(fm_dtype a, fm_dtype b) {
  // a, b of the same precision family; complex wins
  if (is_complex(a)) return a;
  if (is_complex(b)) return complex_of(a);
  return a;
}

static bool is_fft_leaf(const fm_op_s* A) {
  return (A->kind == K_FOURIER || A->kind == K_CIRCULANT || A->kind == K_TOEPLITZ) && A->L > 1 && !A->dense;
}

fm_status natural_out_dtype(const fm_op_s* A, fm_dtype in, fm_dtype* out) {
  switch (A->kind) {
    case K_FOURIER:
      if (!is_float_type(in)) break;
      *out = complex_of(in);
      return FM_OK;
    case K_CIRCULANT:
    case K_TOEPLITZ:
    case K_DIAG:
      if (!is_float_type(in)) break;
      *out = A->real ? in : complex_of(in);
      return FM_OK;
    case K_PARTIAL:
      if (!is_float_type(in)) break;
      *out = in;
      return FM_OK;
    case K_HADAMARD:
      if (A->had_mode == FM_HAD_INT8) {
        if (in != FM_I8) break;
        *out = FM_I32;
        return FM_OK;
      }
      if (A->had_mode == FM_HAD_FP32) {
        if (in != FM_F32 && in != FM_C64) break;
        *out = in;
        return FM_OK;
      }
      if (in != FM_F32) break;
      *out = FM_F32;
      return FM_OK;
    case K_HERMITIAN:
      return natural_out_dtype(A->kids[0], in, out);
    case K_PRODUCT: {
      fm_dtype d = in;
      for (int k = (int)A->kids.size() - 1; k >= 0; --k) FM_TRY(natural_out_dtype(A->kids[k], d, &d));
      *out = d;
      return FM_OK;
    }
    case K_KRON: {
      fm_dtype d = in;
      for (auto* f : A->kids) FM_TRY(natural_out_dtype(f, d, &d));
      *out = d;
      return FM_OK;
    }
    case K_SUM:
    case K_BLOCKS:
    case K_BLKDIAG: {
      fm_dtype r = in;
      bool first = true;
      for (auto* t : A->kids) {
        fm_dtype d;
        FM_TRY(natural_out_dtype(t, in, &d));
        if (first) r = d;
        else if (d != r) {
          if (!is_float_type(d) || !is_float_type(r)) {
            set_error("terms produce incompatible dtypes");
            return FM_ERR_DTYPE;
          }
          r = promote(r, d);
        }
        first = false;
      }
      *out = r;
      return FM_OK;
    }
  }
  set_error("operator does not accept input dtype %d", (int)in);
  return FM_ERR_DTYPE;
}

static int64_t in_len(const fm_op_s* A, bool adj) { return adj ? A->rows : A->cols; }
static int64_t out_len(const fm_op_s* A, bool adj) { return adj ? A->cols : A->rows; }

static View packed_view(void* p, fm_dtype dt, int64_t outer, int64_t n, int64_t inner) {
  View v;
  v.p = p;
  v.dt = dt;
  v.outer = outer;
  v.n = n;
  v.inner = inner;
  v.ostride = n * inner;
  v.ld = outer * n * inner;
  return v;
}

static View temp_view(Ctx& ctx, fm_dtype dt, const View& like, int64_t n, int64_t ncols) {
  const int64_t elems = like.outer * n * like.inner * ncols;
  void* p = ctx.alloc((size_t)elems * dtype_size(dt));
  return packed_view(p, dt, like.outer, n, like.inner);
}

static char* elem_ptr(void* p, fm_dtype dt, int64_t off) { return (char*)p + off * dtype_size(dt); }

// copy / convert / accumulate a whole view (dtype promotion between stages)
static fm_status copy_view(const View& in, const View& out, int64_t ncols, int beta, Ctx& ctx) {
  if (ctx.dry) return FM_OK;
  if (in.dt == FM_I32 && out.dt == FM_I32) {
    if (in.outer != 1 || out.outer != 1 || in.inner != 1 || out.inner != 1) {
      set_error("int32 copy on a strided view");
      return FM_ERR_UNSUPPORTED;
    }
    return i32_copy_launch((const int*)in.p, in.ld, (int*)out.p, out.ld, out.n, ncols, beta, ctx.st);
  }
  if (!is_float_type(in.dt) || !is_float_type(out.dt) || is_double(in.dt) != is_double(out.dt)) {
    set_error("cannot convert dtype %d to %d", (int)in.dt, (int)out.dt);
    return FM_ERR_DTYPE;
  }
  PwArgs a;
  a.ncols = ncols;
  a.outer = out.outer;
  a.inner = out.inner;
  a.n_out = out.n;
  a.in = in.p;
  a.in_ld = in.ld;
  a.in_ostride = in.ostride;
  a.in_cplx = is_complex(in.dt);
  a.out = out.p;
  a.out_ld = out.ld;
  a.out_ostride = out.ostride;
  a.out_cplx = is_complex(out.dt);
  a.beta = beta;
  return pointwise_launch(a, is_double(in.dt), ctx.st);
}

// ------------------------------------------------------------------ FFT-based leaves
struct Fused {
  const fm_op_s* pre_map = nullptr;   // Partial applied as adjoint (scatter) before the transform
  const fm_op_s* pre_diag = nullptr;
  int pre_conj = 0;
  const fm_op_s* post_diag = nullptr;
  int post_conj = 0;
  const fm_op_s* post_map = nullptr;  // Partial applied forward (gather) after the transform
};

// the pass-twiddle tables the tile passes read (fm_device.cuh)
template <typename T>
static const typename Cx<T>::t* tw_table(Ctx& ctx) {
  if constexpr (sizeof(T) == 4) return ctx.tabs->twp32;
  else return ctx.tabs->twp64;
}

template <typename T>
static const typename Cx<T>::t* diag_c(const fm_op_s* D) {
  if constexpr (sizeof(T) == 4) return D->d32;
  else return D->d64;
}
template <typename T>
static const T* diag_r(const fm_op_s* D) {
  if constexpr (sizeof(T) == 4) return D->dr32;
  else return D->dr64;
}

struct FftJob {
  int64_t L = 0;
  const BigPlan* big = nullptr;
  int conv = 0;
  int dir = -1;           // Fourier direction
  const void* spec = nullptr;
  const void* spec_perm = nullptr;
  int spec_conj = 0;
  double scale = 1.0;
  int64_t Lin = 0, Lout = 0;  // lengths of the transform's input and output vectors
  bool real = false;          // operator (with fused diagonals) is real
  int tile = 0, rcap = 0;     // execution plan of the tiles (fm_op_s::tile, rcap)
};

template <typename T>
static void set_pre_post(FftArgs<T>& a, const Fused& F) {
  if (F.pre_map) a.pre_map = F.pre_map->inv;
  if (F.pre_diag) {
    if (F.pre_diag->real) a.pre_dr = diag_r<T>(F.pre_diag);
    else a.pre_dc = diag_c<T>(F.pre_diag);
    a.pre_conj = F.pre_conj;
  }
  if (F.post_diag) {
    if (F.post_diag->real) a.post_dr = diag_r<T>(F.post_diag);
    else a.post_dc = diag_c<T>(F.post_diag);
    a.post_conj = F.post_conj;
  }
  if (F.post_map) a.post_map = F.post_map->inv;
}

template <typename T>
static fm_status run_fft(const FftJob& J, const Fused& F, const View& in, const View& out, int64_t ncols, int beta,
                         Ctx& ctx) {
  typedef typename Cx<T>::t C;
  const bool in_c = is_complex(in.dt), out_c = is_complex(out.dt);
  int in_mode, out_mode;
  int64_t ncu;
  if (!in_c && !out_c) {
    if (!J.real) { set_error("complex operator into a real buffer"); return FM_ERR_DTYPE; }
    in_mode = IO_RP;
    out_mode = IO_RP;
    ncu = (ncols + 1) / 2;
  } else if (!in_c) {
    in_mode = IO_R;
    out_mode = IO_C;
    ncu = ncols;
  } else {
    if (!out_c) { set_error("complex data into a real buffer"); return FM_ERR_DTYPE; }
    in_mode = IO_C;
    out_mode = IO_C;
    ncu = ncols;
  }
  if (in.outer != out.outer || in.inner != out.inner) {
    set_error("fft: input and output views differ in outer/inner");
    return FM_ERR_SHAPE;
  }
  // A small FP64 problem (a few columns of a transform of 2^11 .. 2^13) would occupy only a
  // few CTAs as whole-vector tiles; its two-pass plan with small tiles spreads the FP64
  // work over many SMs.
  const int64_t vec_single = std::max<int64_t>(1, 4096 / J.L);
  const int64_t tiles_single = (ncu * in.outer * in.inner + vec_single - 1) / vec_single;
  const bool small = sizeof(T) == 8 && J.big && J.big->L == J.L && J.L <= fft_max_tile<T>() && tiles_single < 64;
  if (J.L <= fft_max_tile<T>() && !small) {
    if (ctx.dry) return FM_OK;
    FftArgs<T> a;
    a.tile = J.tile;
    a.rcap = J.rcap;
    a.L = J.L;
    a.conv = J.conv;
    a.dir0 = J.conv ? -1 : J.dir;
    a.spec = (const C*)J.spec;
    a.spec_conj = J.spec_conj;
    a.tw = tw_table<T>(ctx);
    a.ncu = ncu;
    a.ncols = ncols;
    a.outer = in.outer;
    a.inner = in.inner;
    a.in = in.p;
    a.in_ld = in.ld;
    a.in_ostride = in.ostride;
    a.in_tstride = in.inner;
    a.in_imod = in.inner;
    a.in_mode = in_mode;
    a.Lin = J.Lin;
    a.out = out.p;
    a.out_ld = out.ld;
    a.out_ostride = out.ostride;
    a.out_tstride = out.inner;
    a.out_imod = out.inner;
    a.out_mode = out_mode;
    a.Lout = J.Lout;
    set_pre_post(a, F);
    a.scale = (T)J.scale;
    a.beta = beta;
    return fft_launch<T>(a, ctx.st);
  }
  // ---- two-pass plan, L = N1 * N2: column DFTs of length N1 (stride N2), twiddles,
  //      row DFTs of length N2 (and, for a convolution, spectrum product, inverse row
  //      DFTs, conjugate twiddles and inverse column DFTs).
  const BigPlan* B = J.big;
  if (!B || B->L != J.L) { set_error("missing two-pass plan for length %lld", (long long)J.L); return FM_ERR_UNSUPPORTED; }
  if (in.outer > 1) {
    for (int64_t o = 0; o < in.outer; ++o) {
      View ii = in, oo = out;
      ii.outer = oo.outer = 1;
      ii.p = elem_ptr(in.p, in.dt, o * in.ostride);
      oo.p = elem_ptr(out.p, out.dt, o * out.ostride);
      FM_TRY(run_fft<T>(J, F, ii, oo, ncols, beta, ctx));
    }
    return FM_OK;
  }
  const int64_t N1 = B->N1, N2 = B->N2, L = J.L, inner = in.inner;
  C* scratch = (C*)ctx.alloc((size_t)ncu * L * inner * sizeof(C));
  if (ctx.dry) return FM_OK;
  const C* twL;
  if constexpr (sizeof(T) == 4) twL = B->tw32;
  else twL = B->tw64;
  const int dirA = J.conv ? -1 : J.dir;
  // pass A
  {
    FftArgs<T> a;
    a.tile = J.tile;
    a.rcap = J.rcap;
    a.small = small ? 1 : 0;
    a.L = N1;
    a.dir0 = dirA;
    a.tw = tw_table<T>(ctx);
    a.ncu = ncu;
    a.ncols = ncols;
    a.outer = 1;
    a.inner = N2 * inner;
    a.in = in.p;
    a.in_ld = in.ld;
    a.in_ostride = 0;
    a.in_tstride = inner;
    a.in_imod = inner;
    a.in_fmul = N2;
    a.in_fdiv = inner;
    a.in_fmod = N2;
    a.in_mode = in_mode;
    a.Lin = J.Lin;
    a.out = scratch;
    a.out_ld = L * inner;
    a.out_ostride = 0;
    a.out_tstride = N2 * inner;
    a.out_imod = N2 * inner;
    a.out_mode = IO_C;
    a.Lout = N1;
    Fused pre = F;
    pre.post_diag = nullptr;
    pre.post_map = nullptr;
    set_pre_post(a, pre);
    a.post_tw = twL;
    a.post_tw_conj = dirA > 0;
    a.tw_mask = L - 1;
    a.tw_div = inner;
    a.tw_mod = N2;
    FM_TRY(fft_launch<T>(a, ctx.st));
  }
  // pass B
  {
    FftArgs<T> a;
    a.tile = J.tile;
    a.rcap = J.rcap;
    a.small = small ? 1 : 0;
    a.L = N2;
    a.tw = tw_table<T>(ctx);
    a.ncu = ncu;
    a.ncols = ncols;
    a.outer = N1;
    a.inner = inner;
    a.in = scratch;
    a.in_ld = L * inner;
    a.in_ostride = N2 * inner;
    a.in_tstride = inner;
    a.in_imod = inner;
    a.in_mode = IO_C;
    a.Lin = N2;
    if (J.conv) {
      a.conv = 1;
      a.dir0 = -1;
      a.spec = (const C*)J.spec_perm;
      a.spec_omod = N1;
      a.spec_conj = J.spec_conj;
      a.out = scratch;
      a.out_ld = L * inner;
      a.out_ostride = N2 * inner;
      a.out_tstride = inner;
      a.out_imod = inner;
      a.out_mode = IO_C;
      a.Lout = N2;
    } else {
      a.dir0 = J.dir;
      a.out = out.p;
      a.out_ld = out.ld;
      a.out_ostride = 0;
      a.out_tstride = inner;
      a.out_imod = inner;
      a.out_fmul = N1;
      a.out_fdiv = inner;
      a.out_fmod = N1;
      a.out_mode = out_mode;
      a.Lout = J.Lout;
      Fused post = F;
      post.pre_diag = nullptr;
      post.pre_map = nullptr;
      set_pre_post(a, post);
      a.scale = (T)J.scale;
      a.beta = beta;
    }
    FM_TRY(fft_launch<T>(a, ctx.st));
  }
  if (!J.conv) return FM_OK;
  // pass C
  {
    FftArgs<T> a;
    a.tile = J.tile;
    a.rcap = J.rcap;
    a.small = small ? 1 : 0;
    a.L = N1;
    a.dir0 = +1;
    a.tw = tw_table<T>(ctx);
    a.ncu = ncu;
    a.ncols = ncols;
    a.outer = 1;
    a.inner = N2 * inner;
    a.in = scratch;
    a.in_ld = L * inner;
    a.in_ostride = 0;
    a.in_tstride = N2 * inner;
    a.in_imod = N2 * inner;
    a.in_mode = IO_C;
    a.Lin = N1;
    a.pre_tw = twL;
    a.pre_tw_conj = 1;
    a.tw_mask = L - 1;
    a.tw_div = inner;
    a.tw_mod = N2;
    a.out = out.p;
    a.out_ld = out.ld;
    a.out_ostride = 0;
    a.out_tstride = inner;
    a.out_imod = inner;
    a.out_fmul = N2;
    a.out_fdiv = inner;
    a.out_fmod = N2;
    a.out_mode = out_mode;
    a.Lout = J.Lout;
    Fused post = F;
    post.pre_diag = nullptr;
    post.pre_map = nullptr;
    set_pre_post(a, post);
    a.scale = (T)J.scale;
    a.beta = beta;
    FM_TRY(fft_launch<T>(a, ctx.st));
  }
  return FM_OK;
}

static bool group_real(const fm_op_s* A, const Fused& F) {
  bool r = A->real;
  if (F.pre_diag && !F.pre_diag->real) r = false;
  if (F.post_diag && !F.post_diag->real) r = false;
  return r;
}

static fm_status exec_fft_leaf(const fm_op_s* A, bool adj, const Fused& F, const View& in, const View& out,
                               int64_t ncols, int beta, Ctx& ctx) {
  FftJob J;
  J.L = A->L;
  J.big = A->big.L ? &A->big : nullptr;
  J.Lin = in_len(A, adj);
  J.Lout = out_len(A, adj);
  J.real = group_real(A, F);
  J.tile = A->tile;
  J.rcap = A->rcap;
  const bool dbl = is_double(in.dt);
  if (A->kind == K_FOURIER) {
    J.conv = 0;
    J.dir = adj ? +1 : -1;
    J.scale = A->ortho ? 1.0 / std::sqrt((double)A->L) : 1.0;
  } else {
    J.conv = 1;
    J.spec = dbl ? (const void*)A->spec64 : (const void*)A->spec32;
    J.spec_perm = dbl ? (const void*)A->spec64_perm : (const void*)A->spec32_perm;
    J.spec_conj = adj ? 1 : 0;
  }
  return dbl ? run_fft<double>(J, F, in, out, ncols, beta, ctx) : run_fft<float>(J, F, in, out, ncols, beta, ctx);
}

// ------------------------------------------------------------------ pointwise leaves
static fm_status exec_pointwise(const fm_op_s* A, bool adj, const View& in, const View& out, int64_t ncols,
                                int beta, Ctx& ctx) {
  if (ctx.dry) return FM_OK;
  PwArgs a;
  a.ncols = ncols;
  a.outer = out.outer;
  a.inner = out.inner;
  a.n_out = out.n;
  a.in = in.p;
  a.in_ld = in.ld;
  a.in_ostride = in.ostride;
  a.in_cplx = is_complex(in.dt);
  a.out = out.p;
  a.out_ld = out.ld;
  a.out_ostride = out.ostride;
  a.out_cplx = is_complex(out.dt);
  a.beta = beta;
  const bool dbl = is_double(in.dt);
  switch (A->kind) {
    case K_DIAG:
      if (A->real) a.dr = dbl ? (const void*)A->dr64 : (const void*)A->dr32;
      else a.dc = dbl ? (const void*)A->d64 : (const void*)A->d32;
      a.d_conj = adj;
      break;
    case K_PARTIAL:
      a.map = adj ? A->inv : A->idx;
      break;
    case K_FOURIER:  // n = 1: identity
    case K_HADAMARD:
      break;
    case K_CIRCULANT:  // n = 1: scalar c0
    case K_TOEPLITZ:
      if (A->real) a.dr = dbl ? (const void*)A->dr64 : (const void*)A->dr32;
      else a.dc = dbl ? (const void*)A->d64 : (const void*)A->d32;
      a.d_conj = adj;
      break;
    default:
      set_error("not a pointwise operator");
      return FM_ERR_INVALID_ARG;
  }
  return pointwise_launch(a, dbl, ctx.st);
}

// ------------------------------------------------------------------ Hadamard
static fm_status exec_hadamard(const fm_op_s* A, const View& in, const View& out, int64_t ncols, int beta,
                               Ctx& ctx) {
  if (A->log2n == 0) {
    if (in.dt == FM_I8) {
      set_error("int8 Hadamard of length 1 is not supported");
      return FM_ERR_UNSUPPORTED;
    }
    return exec_pointwise(A, false, in, out, ncols, beta, ctx);
  }
  if (A->log2n >= 17 && A->had_mode != FM_HAD_BF16 && A->had_mode != FM_HAD_BF16X2) {
    // H_{2^(a+b)} = (H_{2^a} (x) I_{2^b}) (I_{2^a} (x) H_{2^b}): the low 14 index bits as
    // contiguous blocks, then the top bits along the axis of stride 2^14 (in place in the
    // output, or through a scratch column block when accumulating)
    const int lb = 14, la = A->log2n - lb;
    const int64_t nb = 1LL << lb, na = 1LL << la;
    const fm_dtype td = in.dt == FM_I8 ? FM_I32 : in.dt;
    View t = out;
    const size_t mark = ctx.used;
    if (beta || td != out.dt) t = temp_view(ctx, td, out, out.n, ncols);
    fm_op_s hb, ha;  // the two factors (only their length and mode are read)
    hb.kind = ha.kind = K_HADAMARD;
    hb.had_mode = ha.had_mode = A->had_mode;
    hb.log2n = lb;
    ha.log2n = la;
    View i1 = in, o1 = t;
    i1.outer = in.outer * na;
    i1.n = nb;
    i1.ostride = nb * in.inner;
    o1.outer = t.outer * na;
    o1.n = nb;
    o1.ostride = nb * t.inner;
    if (in.outer > 1 && in.ostride != in.n * in.inner) {
      set_error("Hadamard of length 2^%d on a view with a gap between outer blocks", A->log2n);
      return FM_ERR_UNSUPPORTED;
    }
    FM_TRY(exec_hadamard(&hb, i1, o1, ncols, 0, ctx));
    View i2 = t, o2 = out;
    i2.n = o2.n = na;
    i2.inner = nb * t.inner;
    o2.inner = nb * out.inner;
    FM_TRY(exec_hadamard(&ha, i2, o2, ncols, beta, ctx));
    ctx.used = mark;
    return FM_OK;
  }
  FwhtArgs a;
  a.logL = A->log2n;
  a.ncols = ncols;
  a.outer = in.outer;
  a.inner = in.inner;
  a.in = in.p;
  a.in_ld = in.ld;
  a.in_ostride = in.ostride;
  a.in_tstride = in.inner;
  a.out = out.p;
  a.out_ld = out.ld;
  a.out_ostride = out.ostride;
  a.out_tstride = out.inner;
  a.beta = beta;
  a.prefetch = A->tile == 0 ? 1 : 0;
  if (ctx.dry) return FM_OK;
  if (A->had_mode == FM_HAD_BF16 || A->had_mode == FM_HAD_BF16X2)
    return fwht_mma_launch(a, A->had_mode == FM_HAD_BF16X2 ? 1 : 0, ctx.st);
  return fwht_launch(a, in.dt, ctx.st);
}

// ------------------------------------------------------------------ composites
struct Item {
  const fm_op_s* op;
  bool adj;
};

static void flatten(const fm_op_s* A, bool adj, std::vector<Item>& seq) {
  if (A->kind == K_PRODUCT) {
    const int k = (int)A->kids.size();
    if (!adj) for (int i = k - 1; i >= 0; --i) flatten(A->kids[i], adj, seq);
    else for (int i = 0; i < k; ++i) flatten(A->kids[i], adj, seq);
  } else if (A->kind == K_HERMITIAN) {
    flatten(A->kids[0], !adj, seq);
  } else {
    seq.push_back({A, adj});
  }
}

struct Group {
  Item main;
  bool fft = false;
  Fused F;
  int64_t in_n = 0, out_n = 0;
};

static fm_status exec_product(const fm_op_s* A, bool adj, const View& in, const View& out, int64_t ncols, int beta,
                              Ctx& ctx) {
  std::vector<Item> seq;
  flatten(A, adj, seq);
  std::vector<Group> groups;
  size_t i = 0;
  while (i < seq.size()) {
    Group g;
    size_t j = i;
    auto is_fft = [&](size_t k) { return k < seq.size() && is_fft_leaf(seq[k].op); };
    auto is_diag = [&](size_t k) { return k < seq.size() && seq[k].op->kind == K_DIAG; };
    auto is_part = [&](size_t k, bool a) {
      return k < seq.size() && seq[k].op->kind == K_PARTIAL && seq[k].adj == a;
    };
    if (is_part(j, true) && (is_fft(j + 1) || (is_diag(j + 1) && is_fft(j + 2)))) {
      g.F.pre_map = seq[j].op;
      ++j;
    }
    if (is_diag(j) && is_fft(j + 1)) {
      g.F.pre_diag = seq[j].op;
      g.F.pre_conj = seq[j].adj;
      ++j;
    }
    if (is_fft(j)) {
      g.main = seq[j];
      g.fft = true;
      ++j;
      if (is_diag(j)) {
        g.F.post_diag = seq[j].op;
        g.F.post_conj = seq[j].adj;
        ++j;
      }
      if (is_part(j, false)) {
        g.F.post_map = seq[j].op;
        ++j;
      }
    } else {
      g = Group();
      g.main = seq[i];
      j = i + 1;
    }
    g.in_n = g.F.pre_map ? g.F.pre_map->rows : in_len(g.main.op, g.main.adj);
    g.out_n = g.F.post_map ? g.F.post_map->rows : out_len(g.main.op, g.main.adj);
    groups.push_back(g);
    i = j;
  }
  // dtype of each group's output
  View cur = in;
  const size_t mark = ctx.used;
  for (size_t k = 0; k < groups.size(); ++k) {
    const Group& g = groups[k];
    fm_dtype od;
    FM_TRY(natural_out_dtype(g.main.op, cur.dt, &od));
    if (g.F.pre_diag && !g.F.pre_diag->real) od = complex_of(od);
    if (g.F.post_diag && !g.F.post_diag->real) od = complex_of(od);
    if (g.fft && !is_complex(cur.dt) && !group_real(g.main.op, g.F)) od = complex_of(od);
    const bool last = k + 1 == groups.size();
    View dst;
    if (last) {
      dst = out;
    } else {
      dst = temp_view(ctx, od, in, g.out_n, ncols);
    }
    if (g.fft) {
      if (!last || od == out.dt) {
        FM_TRY(exec_fft_leaf(g.main.op, g.main.adj, g.F, cur, dst, ncols, last ? beta : 0, ctx));
      } else {
        View tmp = temp_view(ctx, od, in, g.out_n, ncols);
        FM_TRY(exec_fft_leaf(g.main.op, g.main.adj, g.F, cur, tmp, ncols, 0, ctx));
        FM_TRY(copy_view(tmp, out, ncols, beta, ctx));
      }
    } else {
      FM_TRY(exec(g.main.op, g.main.adj, cur, dst, ncols, last ? beta : 0, ctx));
    }
    cur = dst;
  }
  ctx.used = mark;
  return FM_OK;
}

static fm_status exec_kron(const fm_op_s* A, bool adj, const View& in, const View& out, int64_t ncols, int beta,
                           Ctx& ctx) {
  const int k = (int)A->kids.size();
  if (k == 1) return exec(A->kids[0], adj, in, out, ncols, beta, ctx);
  const bool in_packed = in.outer == 1 || in.ostride == in.n * in.inner;
  const bool out_packed = out.outer == 1 || out.ostride == out.n * out.inner;
  if (!in_packed || !out_packed) {
    for (int64_t o = 0; o < in.outer; ++o) {
      View ii = in, oo = out;
      ii.outer = oo.outer = 1;
      ii.p = elem_ptr(in.p, in.dt, o * in.ostride);
      oo.p = elem_ptr(out.p, out.dt, o * out.ostride);
      FM_TRY(exec_kron(A, adj, ii, oo, ncols, beta, ctx));
    }
    return FM_OK;
  }
  std::vector<int64_t> cur(k);
  for (int j = 0; j < k; ++j) cur[j] = in_len(A->kids[j], adj);
  const size_t mark = ctx.used;
  View src = in;
  src.ostride = in.n * in.inner;
  // Hadamard outermost and Fourier innermost on complex64 columns: both in one fused pass
  // (the mode products commute), then the middle factors as usual
  const fm_op_s* f0 = A->kids[0];
  const fm_op_s* fl = A->kids[k - 1];
  int la = 0, lb = 0;
  while ((1LL << lb) < fl->L) ++lb;
  la = f0->log2n;
  const bool fuse = f0->kind == K_HADAMARD && f0->had_mode == FM_HAD_FP32 && fl->kind == K_FOURIER &&
                    in.dt == FM_C64 && out.dt == FM_C64 && in.outer == 1 && in.inner == 1 && out.outer == 1 &&
                    out.inner == 1 && kron_hf_ok(la, lb);
  int jfirst = 0, jlast = k;
  if (fuse) {
    const int64_t N = in.n;
    const int64_t nmid = N >> (la + lb);
    View d = out;
    if (k > 2) {
      d = packed_view(ctx.alloc((size_t)N * ncols * sizeof(float2)), FM_C64, 1, N, 1);
      d.ld = N;
    }
    if (!ctx.dry) {
      KronHFArgs h;
      h.in = reinterpret_cast<const float2*>(in.p);
      h.out = reinterpret_cast<float2*>(d.p);
      h.in_ld = in.ld;
      h.out_ld = d.ld;
      h.nmid = nmid;
      h.ntiles = ncols * nmid;
      h.sa = nmid << lb;
      h.dir = adj ? +1 : -1;
      h.scale = fl->ortho ? (float)(1.0 / std::sqrt((double)fl->L)) : 1.f;
      h.beta = k > 2 ? 0 : beta;
      h.tw = tw_table<float>(ctx);
      h.pair = A->tile;   // the Kron operator's plan: one CTA, a pair or a quad of CTAs per tile
      FM_TRY(kron_hf_launch(h, la, lb, ctx.st));
    }
    if (k == 2) {
      ctx.used = mark;
      return FM_OK;
    }
    src = d;
    src.ostride = N;
    jfirst = 1;
    jlast = k - 1;
  }
  for (int j = jfirst; j < jlast; ++j) {
    const fm_op_s* f = A->kids[j];
    int64_t outer = in.outer, inner = in.inner;
    for (int l = 0; l < j; ++l) outer *= cur[l];
    for (int l = j + 1; l < k; ++l) inner *= cur[l];
    fm_dtype od;
    FM_TRY(natural_out_dtype(f, src.dt, &od));
    const int64_t nout = out_len(f, adj);
    View s = src;
    s.outer = outer;
    s.inner = inner;
    s.n = cur[j];
    s.ostride = cur[j] * inner;
    const bool last = j + 1 == jlast;
    View d;
    if (last) {
      // natural_out_dtype(A) == out.dt here: the caller promotes otherwise
      d = out;
      d.outer = outer;
      d.inner = inner;
      d.n = nout;
      d.ostride = nout * inner;
      FM_TRY(exec(f, adj, s, d, ncols, beta, ctx));
    } else {
      d = packed_view(ctx.alloc((size_t)outer * nout * inner * ncols * dtype_size(od)), od, outer, nout, inner);
      d.ld = outer * nout * inner;
      FM_TRY(exec(f, adj, s, d, ncols, 0, ctx));
    }
    cur[j] = nout;
    // the next factor sees the whole (packed) column again
    src = d;
    src.ld = d.ld;
  }
  ctx.used = mark;
  return FM_OK;
}

fm_status exec(const fm_op_s* A, bool adj, const View& in, const View& out, int64_t ncols, int beta, Ctx& ctx) {
  if (ncols == 0) return FM_OK;
  fm_dtype nd;
  FM_TRY(natural_out_dtype(A, in.dt, &nd));
  if (nd != out.dt && A->kind != K_PRODUCT) {
    // compute in the natural type, then promote into the caller's buffer
    const size_t mark = ctx.used;
    View t = temp_view(ctx, nd, out, out.n, ncols);
    FM_TRY(exec(A, adj, in, t, ncols, 0, ctx));
    FM_TRY(copy_view(t, out, ncols, beta, ctx));
    ctx.used = mark;
    return FM_OK;
  }
  if (A->dense && is_complex(in.dt) && in.dt == out.dt && in.outer == 1 && in.inner == 1 && out.outer == 1 &&
      out.inner == 1) {
    if (ctx.dry) return FM_OK;
    return dense_apply(A, adj, in.p, in.ld, out.p, out.ld, ncols, is_double(in.dt), beta, ctx.st);
  }
  switch (A->kind) {
    case K_FOURIER:
    case K_CIRCULANT:
    case K_TOEPLITZ:
      if (A->L <= 1) return exec_pointwise(A, adj, in, out, ncols, beta, ctx);
      return exec_fft_leaf(A, adj, Fused(), in, out, ncols, beta, ctx);
    case K_HADAMARD:
      return exec_hadamard(A, in, out, ncols, beta, ctx);
    case K_DIAG:
    case K_PARTIAL:
      return exec_pointwise(A, adj, in, out, ncols, beta, ctx);
    case K_HERMITIAN:
      return exec(A->kids[0], !adj, in, out, ncols, beta, ctx);
    case K_PRODUCT:
      return exec_product(A, adj, in, out, ncols, beta, ctx);
    case K_SUM: {
      for (size_t k = 0; k < A->kids.size(); ++k)
        FM_TRY(exec(A->kids[k], adj, in, out, ncols, k == 0 ? beta : 1, ctx));
      return FM_OK;
    }
    case K_BLKDIAG: {
      int64_t ioff = 0, ooff = 0;
      for (auto* b : A->kids) {
        View ii = in, oo = out;
        ii.n = in_len(b, adj);
        oo.n = out_len(b, adj);
        ii.p = elem_ptr(in.p, in.dt, ioff * in.inner);
        oo.p = elem_ptr(out.p, out.dt, ooff * out.inner);
        FM_TRY(exec(b, adj, ii, oo, ncols, beta, ctx));
        ioff += ii.n;
        ooff += oo.n;
      }
      return FM_OK;
    }
    case K_KRON:
      return exec_kron(A, adj, in, out, ncols, beta, ctx);
    case K_BLOCKS: {
      // output segment i = sum_j B_ij (input segment j); adjoint: segment j = sum_i B_ij^H (segment i)
      const int R = A->blk_r, Cn = A->blk_c;
      const int no = adj ? Cn : R, ni = adj ? R : Cn;
      int64_t ooff = 0;
      for (int a = 0; a < no; ++a) {
        int64_t ioff = 0;
        for (int b = 0; b < ni; ++b) {
          const fm_op_s* B = adj ? A->kids[b * Cn + a] : A->kids[a * Cn + b];
          View ii = in, oo = out;
          ii.n = in_len(B, adj);
          oo.n = out_len(B, adj);
          ii.p = elem_ptr(in.p, in.dt, ioff * in.inner);
          oo.p = elem_ptr(out.p, out.dt, ooff * out.inner);
          FM_TRY(exec(B, adj, ii, oo, ncols, b == 0 ? beta : 1, ctx));
          ioff += ii.n;
        }
        ooff += out_len(adj ? A->kids[a] : A->kids[a * Cn], adj);
      }
      return FM_OK;
    }
  }
  set_error("unknown operator kind");
  return FM_ERR_INVALID_ARG;
}

// ------------------------------------------------------------------ construction helpers
fm_status make_big_plan(int64_t L, BigPlan* plan, cudaStream_t st) {
  int lg = 0;
  while ((1LL << lg) < L) ++lg;
  plan->L = L;
  plan->N1 = 1LL << (lg / 2);
  plan->N2 = L / plan->N1;
  FM_CUDA(cudaMalloc(&plan->tw32, (size_t)L * sizeof(float2)));
  FM_CUDA(cudaMalloc(&plan->tw64, (size_t)L * sizeof(double2)));
  return twiddle_launch(L, plan->tw32, plan->tw64, st);
}

void free_big_plan(BigPlan* plan) {
  if (plan->tw32) cudaFree(plan->tw32);
  if (plan->tw64) cudaFree(plan->tw64);
  plan->tw32 = nullptr;
  plan->tw64 = nullptr;
  plan->L = 0;
}

fm_status exec_dft(int64_t L, const BigPlan* big, int dir, const View& in, int64_t lin, const View& out,
                   int64_t ncols, double scale, Ctx& ctx) {
  if (!is_complex(in.dt) || in.dt != out.dt) {
    set_error("exec_dft: complex views of one precision expected");
    return FM_ERR_DTYPE;
  }
  FftJob J;
  J.L = L;
  J.big = big && big->L == L ? big : nullptr;
  J.conv = 0;
  J.dir = dir;
  J.Lin = lin;
  J.Lout = L;
  J.scale = scale;
  J.real = false;
  return is_double(in.dt) ? run_fft<double>(J, Fused(), in, out, ncols, 0, ctx)
                          : run_fft<float>(J, Fused(), in, out, ncols, 0, ctx);
}

fm_status construction_fft64(const double2* in, double2* out, int64_t L, const BigPlan* big, cudaStream_t st) {
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  Ctx ctx;
  ctx.st = st;
  FM_TRY(device_tables(dev, &ctx.tabs));
  FftJob J;
  J.L = L;
  J.big = big;
  J.conv = 0;
  J.dir = -1;
  J.Lin = L;
  J.Lout = L;
  View vi = packed_view((void*)in, FM_C128, 1, L, 1);
  View vo = packed_view(out, FM_C128, 1, L, 1);
  ctx.dry = true;
  FM_TRY(run_fft<double>(J, Fused(), vi, vo, 1, 0, ctx));
  void* ws = nullptr;
  if (ctx.peak) FM_CUDA(cudaMalloc(&ws, ctx.peak));
  ctx.dry = false;
  ctx.base = (char*)ws;
  ctx.used = 0;
  fm_status s = run_fft<double>(J, Fused(), vi, vo, 1, 0, ctx);
  if (ws) {
    cudaStreamSynchronize(st);
    cudaFree(ws);
  }
  return s;
}

}  // namespace fm
