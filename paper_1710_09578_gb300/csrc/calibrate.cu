// Calibration of the two-pass split of long transforms (fm_calibrate, fm_set_split).
//
// The paper's calibration (Sec. 2.1.3) benchmarks the fast transforms of an operator and
// stores what it finds for later decisions.  Here the decision is the split L = N1 x N2
// of a transform longer than one tile: the column pass (length N1, stride N2) and the row
// pass (length N2, with the spectrum product for a convolution) cost differently, and the
// cheapest split depends on the operator and the column count.  The candidates are timed
// on the operator as a whole (forward + adjoint, CUDA events) and the best one is kept.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "fm_internal.h"

namespace fm {
namespace {

__global__ void spec_permute_kernel(const double2* s64, double2* p64, float2* p32, int64_t L, int64_t N1,
                                    int64_t N2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = s64[k];
    const int64_t k1 = k % N1, k2 = k / N1;
    p64[k1 * N2 + k2] = v;
    p32[k1 * N2 + k2] = make_float2((float)v.x, (float)v.y);
  }
}

int ilog2_64(int64_t x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

// Transforms whose two-pass plan is used for full-size work (longer than one FP64 tile;
// the shorter plans only serve small FP64 problems and keep their default split).
void collect(fm_op_s* A, std::vector<fm_op_s*>& out) {
  if (!A) return;
  if ((A->kind == K_FOURIER || A->kind == K_CIRCULANT || A->kind == K_TOEPLITZ) && A->big.L > 8192) {
    if (std::find(out.begin(), out.end(), A) == out.end()) out.push_back(A);
  }
  for (fm_op_s* k : A->kids) collect(k, out);
}

// Every FFT leaf (Fourier, Circulant, Toeplitz) whose tiles have a plan to choose.
void collect_fft(fm_op_s* A, std::vector<fm_op_s*>& out) {
  if (!A) return;
  if ((A->kind == K_FOURIER || A->kind == K_CIRCULANT || A->kind == K_TOEPLITZ) && A->L > 1 && !A->dense) {
    if (std::find(out.begin(), out.end(), A) == out.end()) out.push_back(A);
  }
  for (fm_op_s* k : A->kids) collect_fft(k, out);
}

// Kron operators whose outer Hadamard and inner Fourier factors run as one fused pass.
void collect_kron(fm_op_s* A, std::vector<fm_op_s*>& out) {
  if (!A) return;
  if (A->kind == K_KRON && A->kids.size() >= 2 && A->kids[0]->kind == K_HADAMARD &&
      A->kids[0]->had_mode == FM_HAD_FP32 && A->kids.back()->kind == K_FOURIER) {
    if (std::find(out.begin(), out.end(), A) == out.end()) out.push_back(A);
  }
  for (fm_op_s* k : A->kids) collect_kron(k, out);
}

// Hadamard leaves long enough for the long-column kernels (n >= 2^15, FP32 or int8 input).
void collect_had(fm_op_s* A, std::vector<fm_op_s*>& out) {
  if (!A) return;
  if (A->kind == K_HADAMARD && A->log2n >= 15 && (A->had_mode == FM_HAD_FP32 || A->had_mode == FM_HAD_INT8)) {
    if (std::find(out.begin(), out.end(), A) == out.end()) out.push_back(A);
  }
  for (fm_op_s* k : A->kids) collect_had(k, out);
}

void signature(const fm_op_s* A, std::string& out) {
  static const char* names[] = {"F", "C", "T", "H", "D", "P", "Prod", "Sum", "BlkDiag", "Kron", "Herm", "Blocks"};
  out += names[A->kind];
  out += "[" + std::to_string(A->rows) + "x" + std::to_string(A->cols) + (A->real ? "r" : "c");
  if (A->kind == K_HADAMARD) out += ",m" + std::to_string((int)A->had_mode);
  if (A->kind == K_FOURIER && A->ortho) out += ",o";
  if (A->kind == K_BLOCKS) out += "," + std::to_string(A->blk_r) + "x" + std::to_string(A->blk_c);
  out += "]";
  if (!A->kids.empty()) {
    out += "(";
    for (size_t i = 0; i < A->kids.size(); ++i) {
      if (i) out += ",";
      signature(A->kids[i], out);
    }
    out += ")";
  }
}

bool split_ok(int64_t L, int64_t n1) {
  if (n1 < 32 || (n1 & (n1 - 1)) || L % n1) return false;
  const int64_t n2 = L / n1;
  return n1 <= 8192 && n2 >= 32 && n2 <= 8192;
}

fm_status set_leaf_split(fm_op_s* A, int64_t n1, cudaStream_t st) {
  const int64_t L = A->big.L;
  if (n1 == A->big.N1) return FM_OK;
  A->big.N1 = n1;
  A->big.N2 = L / n1;
  if (A->spec64 && A->spec64_perm) {
    int64_t blocks = (L + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    spec_permute_kernel<<<(unsigned)blocks, 256, 0, st>>>(A->spec64, A->spec64_perm, A->spec32_perm, L, n1, L / n1);
    FM_TRY(after_launch("spec_permute_kernel"));
  }
  return FM_OK;
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" {

fm_status fm_set_split(fm_op A, int64_t L, int64_t n1, void* stream) {
  clear_error();
  if (!A) { set_error("null operator"); return FM_ERR_INVALID_ARG; }
  if (n1 == 0) n1 = (int64_t)1 << (ilog2_64(L) / 2);
  if (!split_ok(L, n1)) {
    set_error("split %lld x %lld of %lld: N1 and N2 must be powers of two in [2^5, 2^13]", (long long)n1,
              (long long)(n1 ? L / n1 : 0), (long long)L);
    return FM_ERR_INVALID_ARG;
  }
  std::vector<fm_op_s*> leaves;
  collect(A, leaves);
  cudaStream_t st = (cudaStream_t)stream;
  for (fm_op_s* leaf : leaves)
    if (leaf->big.L == L) FM_TRY(set_leaf_split(leaf, n1, st));
  FM_CUDA(cudaStreamSynchronize(st));
  return FM_OK;
}

fm_status fm_set_plan(fm_op A, int64_t L, int32_t kind, int64_t value, void* stream) {
  clear_error();
  if (!A) { set_error("null operator"); return FM_ERR_INVALID_ARG; }
  if (kind == 0) return fm_set_split(A, L, value, stream);
  if ((kind == 1 && (value < 0 || value > 4)) || (kind == 2 && value != 0 && value != 3) ||
      (kind == 3 && (value < 0 || value > 3)) || (kind == 5 && (value < 0 || value > 1)) || kind < 0 || kind == 4 ||
      kind > 5) {
    set_error("plan setting %d = %lld: tile shape 0..4, radix cap 0 or 3, fused Kron pass 0..3, Hadamard 0..1", kind,
              (long long)value);
    return FM_ERR_INVALID_ARG;
  }
  if (kind == 5) {
    std::vector<fm_op_s*> hl;
    collect_had(A, hl);
    for (fm_op_s* h : hl)
      if (h->rows == L) h->tile = (int)value;
    return FM_OK;
  }
  if (kind == 3) {
    std::vector<fm_op_s*> kr;
    collect_kron(A, kr);
    for (fm_op_s* k : kr)
      if (k->rows == L) k->tile = (int)value;
    return FM_OK;
  }
  std::vector<fm_op_s*> fl;
  collect_fft(A, fl);
  for (fm_op_s* leaf : fl)
    if (leaf->L == L) (kind == 1 ? leaf->tile : leaf->rcap) = (int)value;
  return FM_OK;
}

fm_status fm_signature(fm_op A, char* buf, int32_t len) {
  clear_error();
  if (!A || !buf || len < 1) { set_error("bad argument"); return FM_ERR_INVALID_ARG; }
  std::string sgn;
  signature(A, sgn);
  if ((int64_t)sgn.size() + 1 > len) { set_error("signature needs %zu bytes", sgn.size() + 1); return FM_ERR_SHAPE; }
  std::memcpy(buf, sgn.c_str(), sgn.size() + 1);
  return FM_OK;
}

fm_status fm_calibrate(fm_op A, int64_t ncols, fm_dtype dt, void* stream, fm_tune_entry* report,
                       int32_t max_entries, int32_t* n_entries) {
  clear_error();
  if (n_entries) *n_entries = 0;
  if (!A || ncols <= 0) { set_error("bad argument"); return FM_ERR_INVALID_ARG; }
  if (dt != FM_F32 && dt != FM_F64 && dt != FM_C64 && dt != FM_C128) { set_error("calibration dtype"); return FM_ERR_DTYPE; }
  std::vector<fm_op_s*> leaves, fleaves, krons;
  collect(A, leaves);
  collect_fft(A, fleaves);
  collect_kron(A, krons);
  if (leaves.empty() && fleaves.empty() && krons.empty()) return FM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const fm_dtype cdt = complex_of(dt);
  const size_t esz = (size_t)dtype_size(cdt);
  void *X = nullptr, *Y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fm_status s = FM_OK;
  auto cleanup = [&]() {
    if (X) cudaFree(X);
    if (Y) cudaFree(Y);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&X, esz * (size_t)A->cols * ncols) != cudaSuccess ||
      cudaMalloc(&Y, esz * (size_t)A->rows * ncols) != cudaSuccess) {
    cleanup();
    set_error("calibration: no memory for %lld probe columns", (long long)ncols);
    return FM_ERR_OOM;
  }
  cudaMemsetAsync(X, 0, esz * (size_t)A->cols * ncols, st);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_once = [&](float* ms) -> fm_status {
    // one warm-up, then the mean of three forward + adjoint pairs
    FM_TRY(fm_forward(A, X, A->cols, cdt, Y, A->rows, cdt, ncols, st));
    FM_TRY(fm_backward(A, Y, A->rows, cdt, X, A->cols, cdt, ncols, st));
    FM_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) {
      FM_TRY(fm_forward(A, X, A->cols, cdt, Y, A->rows, cdt, ncols, st));
      FM_TRY(fm_backward(A, Y, A->rows, cdt, X, A->cols, cdt, ncols, st));
    }
    FM_CUDA(cudaEventRecord(e1, st));
    FM_CUDA(cudaEventSynchronize(e1));
    FM_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= 3.f;
    return FM_OK;
  };
  int32_t done = 0;
  for (fm_op_s* leaf : leaves) {
    const int64_t L = leaf->big.L;
    const int lg = ilog2_64(L);
    std::vector<int64_t> cand;
    for (int e : {lg / 2, lg / 2 - 1, lg / 2 + 1, 6, 5, 7, lg - 13, lg - 12}) {
      const int64_t n1 = (int64_t)1 << std::max(e, 0);
      if (split_ok(L, n1) && std::find(cand.begin(), cand.end(), n1) == cand.end()) cand.push_back(n1);
    }
    const int64_t start = leaf->big.N1;
    int64_t best = start;
    float best_ms = 0.f;
    fm_tune_entry ent = {};
    ent.L = L;
    for (int64_t n1 : cand) {
      if (ent.ncand >= 8) break;
      s = set_leaf_split(leaf, n1, st);
      float ms = 0.f;
      if (s == FM_OK) s = time_once(&ms);
      if (s != FM_OK) break;
      ent.cand_n1[ent.ncand] = n1;
      ent.ms[ent.ncand] = ms;
      ent.ncand++;
      if (best_ms == 0.f || ms < best_ms) {
        best_ms = ms;
        best = n1;
      }
    }
    fm_status s2 = set_leaf_split(leaf, s == FM_OK ? best : start, st);
    if (s == FM_OK) s = s2;
    if (s != FM_OK) break;
    ent.n1 = best;
    ent.kind = 0;
    if (report && done < max_entries) report[done] = ent;
    ++done;
  }
  // the plan of each FFT leaf's tiles (tile shape of strided views, then the radix cap), and of
  // each fused Kron pass (one CTA, a pair or a quad of CTAs per tile)
  struct Setting {
    fm_op_s* op;
    int kind;
  };
  std::vector<Setting> settings;
  for (fm_op_s* leaf : fleaves) settings.push_back({leaf, 1}), settings.push_back({leaf, 2});
  for (fm_op_s* k : krons) settings.push_back({k, 3});
  for (const Setting& set : settings) {
    if (s != FM_OK) break;
    {
      fm_op_s* leaf = set.op;
      const int kind = set.kind;
      int* field = kind == 2 ? &leaf->rcap : &leaf->tile;
      const std::vector<int> cand = kind == 1 ? std::vector<int>{0, 1, 2, 3, 4}
                                  : kind == 2 ? std::vector<int>{0, 3} : std::vector<int>{0, 1, 2, 3};
      const int start = *field;
      int best = start;
      float best_ms = 0.f;
      fm_tune_entry ent = {};
      ent.L = kind == 3 ? leaf->rows : leaf->L;
      ent.kind = kind;
      for (int c : cand) {
        *field = c;
        float ms = 0.f;
        s = time_once(&ms);
        if (s != FM_OK) break;
        ent.cand_n1[ent.ncand] = c;
        ent.ms[ent.ncand] = ms;
        ent.ncand++;
        if (best_ms == 0.f || ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
      *field = s == FM_OK ? best : start;
      ent.n1 = *field;
      if (report && done < max_entries) report[done] = ent;
      ++done;
    }
  }
  if (s == FM_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("calibration: %s", cudaGetErrorString(e));
      s = FM_ERR_CUDA;
    }
  }
  cleanup();
  if (n_entries) *n_entries = done;
  return s;
}

}  // extern "C"
