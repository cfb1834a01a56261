// Executor: runs a plan's contraction sequence on the GPU.
//
// Per batch of 2^batch_log2 bitstrings: fill the projection leaves from the
// bitstrings (Sec. 3.1.1), then for every slice id (Sec. 3.1 slicing) run the
// steps in tree post-order (bit-permute of the operands that need it, batched
// complex GEMM), with the root step's epilogue adding its result in FP64 to
// the batch accumulator (the cross-slice sum, fixed ascending slice order).
// The accumulator is finally mapped to bitstring order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "executor.h"
#include "kernels.cuh"
#include "gemm_tc.cuh"
#include "traj.cuh"
#include "splitk.h"

namespace tnq {

tnq_status cuda_fail(cudaError_t e, const char* what) {
  return fail(TNQ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TNQ_CUDA(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

int timing_begin(Ctx* ctx) {
  if (!ctx->timing) return -1;
  size_t need = ctx->pending.size() * 2 + 2;
  while (ctx->ev_pool.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    ctx->ev_pool.push_back(e);
  }
  int slot = (int)ctx->pending.size() * 2;
  cudaEventRecord(ctx->ev_pool[slot], ctx->stream);
  return slot;
}

void timing_end(Ctx* ctx, int slot, const KernelRecord& r) {
  if (slot < 0) return;
  cudaEventRecord(ctx->ev_pool[slot + 1], ctx->stream);
  ctx->pending.push_back({slot, r});
}

tnq_status timing_collect(Ctx* ctx) {
  for (auto& pr : ctx->pending) {
    float ms = 0;
    cudaError_t e = cudaEventElapsedTime(&ms, ctx->ev_pool[pr.first], ctx->ev_pool[pr.first + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    KernelRecord r = pr.second;
    r.ms = ms;
    ctx->records.push_back(r);
  }
  ctx->pending.clear();
  return TNQ_OK;
}

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int tc_mode_a(int prec) {
  switch (prec) {
    case TNQ_PREC_TF32: return PM_AEXP_TF32;
    case TNQ_PREC_TF32X3: return PM_AEXP_TF32X3;
    case TNQ_PREC_BF16X3: return PM_AEXP_BF16X3;
  }
  return PM_AEXP_F32;
}
int tc_mode_b(int prec) {
  switch (prec) {
    case TNQ_PREC_TF32: return PM_B_TF32;
    case TNQ_PREC_TF32X3: return PM_B_TF32X3;
    case TNQ_PREC_BF16X3: return PM_B_BF16X3;
  }
  return PM_C64;
}

// Bytes of one converted operand half (hi or lo) for n complex elements.
size_t a_half_bytes(int prec, size_t n) { return prec == TNQ_PREC_BF16X3 ? 8 * n : 16 * n; }
size_t b_half_bytes(int prec, size_t n) { return prec == TNQ_PREC_BF16X3 ? 4 * n : 8 * n; }

struct StepOperands {
  const void* a0 = nullptr;
  const void* a1 = nullptr;
  const void* b0 = nullptr;
  const void* b1 = nullptr;
};

cudaError_t perm(Ctx* ctx, const PermDesc& d, const void* src, void* dst0, void* dst1, int slice_id,
               double bytes) {
  KernelRecord r{0, ctx->cur_step, 0, 0, 0, 0, 0.0, bytes, 0.f};
  int slot = timing_begin(ctx);
  cudaError_t e = launch_permute(d, src, dst0, dst1, slice_id, ctx->sm_count, ctx->stream);
  timing_end(ctx, slot, r);
  ctx->launches++;
  return e;
}

// Projection leaves of a bound plan: they sit one after another at equal
// stride (same rank), leaf j reading bitstring-row entry proj_src[j].
struct ProjLeaves {
  char* base = nullptr;
  size_t stride = 0;
  int n_proj = 0, n_open = 0, row_len = 0;
  const int* tab = nullptr;
};

ProjLeaves proj_leaves(const Plan* p, char* ws) {
  ProjLeaves r;
  const int L = p->tree.n_leaves;
  int first = -1;
  for (int i = 0; i < L; ++i)
    if (p->net.leaves[i].kind == LEAF_PROJ) {
      first = i;
      break;
    }
  r.n_proj = (int)p->net.proj_src.size();
  r.n_open = (int)p->net.open_qubits.size();
  r.row_len = p->net.row_len;
  r.tab = reinterpret_cast<const int*>(ws + p->ws_qtab);
  if (first >= 0) {
    r.base = ws + p->tensors[first].offset;
    r.stride = first + 1 < L ? p->tensors[first + 1].offset - p->tensors[first].offset : 0;
  }
  return r;
}

cudaError_t fill_projections(Ctx* ctx, const ProjLeaves& pl, int w, const int8_t* bits, int64_t nv, int* err) {
  ctx->launches++;
  return launch_proj_fill(pl.base, pl.stride, pl.n_proj, pl.n_open, pl.tab, pl.row_len, w, bits, nv, err,
                          ctx->stream);
}

// Root positions of the batch labels (bit j of the bitstring index) and of
// the open qubits' labels (in increasing qubit order).
void root_positions(const Plan* p, std::vector<int>* bpos, std::vector<int>* opos) {
  const auto& rl = p->tensors[p->root].labels;
  auto at = [&](int l) { return int(std::find(rl.begin(), rl.end(), l) - rl.begin()); };
  bpos->clear();
  opos->clear();
  for (int l : p->net.batch_labels) bpos->push_back(at(l));
  for (int l : p->net.open_labels) opos->push_back(at(l));
}

// Host-side check of host bitstrings: -1 exactly at the open qubits, 0/1 elsewhere.
bool host_bits_ok(const Plan* p, int64_t n_bs, const int8_t* bits) {
  const int rl = p->net.row_len;
  std::vector<char> open(rl, 0);
  for (int q : p->net.open_qubits) open[q] = 1;
  for (int64_t b = 0; b < n_bs; ++b)
    for (int q = 0; q < rl; ++q) {
      const int8_t x = bits[b * rl + q];
      if (open[q] ? x != -1 : (x != 0 && x != 1)) return false;
    }
  return true;
}

// Prepare operands (permute / convert) and run one batched complex GEMM.
tnq_status run_gemm_step(Ctx* ctx, const void* a_src, const std::vector<int>& a_labels, bool perm_a,
                         const void* b_src, const std::vector<int>& b_labels, bool perm_b,
                         const std::vector<int>& a_req, const std::vector<int>& b_req,
                         const std::vector<int>& slice_labels, int slice_id, int nH, int nM, int nN, int nK,
                         char* scratch_a, char* scratch_b, void* C, void* acc, int* err, void* part,
                         size_t scratch_a_bytes, int choice = -1) {
  // Small, skinny or K-degenerate steps run on the CUDA cores in FP32 whatever
  // the mode: they are launch- or bandwidth-bound and a tensor-core tile would
  // idle.  An autotuned choice (0 CUDA cores, 1 tensor cores) overrides the rule.
  const double work = std::ldexp(1.0, nH + nM + nN + nK);
  const bool tc_ok = ctx->precision != TNQ_PREC_FP32 && tc_gemm_supported(1 << nM, 1 << nN, 1 << nK, ctx->precision);
  const bool use_tc = choice == 1 ? tc_ok
                      : choice == 0 ? false
                                    : tc_ok && !skinny(nM, nN, nK) && work >= ctx->tc_min_work;
  const size_t out_elems = size_t(1) << (nH + nM + nN);
  const int prec = use_tc ? ctx->precision : TNQ_PREC_FP32;
  StepOperands op;
  PermDesc d;
  const int ns = (int)slice_labels.size();
  // Tall-skinny steps in the tensor-core modes: the large operand is gathered,
  // split and multiplied on the tensor cores in one kernel (choice 2, and the
  // default where the shape qualifies).
  const int n_small = std::min(nM, nN), n_big = std::max(nM, nN);
  // Long-K tall-skinny steps expand the small operand into scratch A (after
  // the small operand itself when that one is permuted into scratch A)
  const size_t tr_used = (nM <= nN && perm_a) ? ((8 * (size_t(1) << a_req.size()) + 4095) & ~size_t(4095)) : 0;
  char* tr_scratch = scratch_a + tr_used;
  const size_t tr_avail = scratch_a_bytes > tr_used ? scratch_a_bytes - tr_used : 0;
  const bool tc_rows_ok = choice != 0 && choice != 1 && ctx->precision != TNQ_PREC_FP32 && n_small <= 7 &&
                          !use_dot(nM, nN, nK) &&
                          tc_rows_supported(1 << n_small, 1 << n_big, 1 << nK, 1 << nH, n_big + nH, ctx->precision) &&
                          tc_rows_scratch_bytes(1 << n_small, 1 << nK, 1 << nH, ctx->precision) <= tr_avail;
  if (tc_rows_ok || (!use_tc && (rows_capable(nM, nN) || use_dot(nM, nN, nK)) && part)) {
    // bandwidth-bound skinny step: complex64 operands in [h][m|n][k] order
    // The large operand of a short-K rows step is read in place (fused gather)
    // instead of being permuted first.
    const bool small_is_a = nM <= nN;
    const bool gather = tc_rows_ok || (!use_dot(nM, nN, nK) && nK <= 5 && (small_is_a ? perm_b : perm_a));
    // Dot steps read an operand in place when its stored layout starts with at
    // least 2^5 K values in the required K order (one contiguous run) and keeps
    // every K bit above the run in K order too (the kernel steps its K offset
    // by adding in the deposited domain, which needs increasing positions).
    auto inplace_dot = [&](const void* src, const std::vector<int>& st, const std::vector<int>& req, DotOp* d) {
      if (!use_dot(nM, nN, nK) || nK > 40 || (int)req.size() - nK > 24) return false;
      auto spos = [&](int l) { return int(std::find(st.begin(), st.end(), l) - st.begin()); };
      *d = DotOp{};
      d->nk = nK;
      d->kmask = 0;
      for (int j = 0; j < nK; ++j) {
        const int q = spos(req[j]);
        if (q >= (int)st.size() || (j < 5 && q != j) || (j > 0 && q <= d->kpos[j - 1])) return false;
        d->kpos[j] = (signed char)q;
        d->kmask |= 1ull << q;
      }
      d->nrow = (int)req.size() - nK;
      for (int j = 0; j < d->nrow; ++j) {
        const int q = spos(req[nK + j]);
        if (q >= (int)st.size()) return false;
        d->rowpos[j] = (signed char)q;
      }
      size_t soff = 0;
      for (int j = 0; j < ns; ++j) {
        const int q = spos(slice_labels[j]);
        if (q < (int)st.size() && ((slice_id >> j) & 1)) soff |= size_t(1) << q;
      }
      d->p = reinterpret_cast<const float2*>(src) + soff;
      return true;
    };
    DotOp dot_a, dot_b;
    const bool inpl_a = perm_a && inplace_dot(a_src, a_labels, a_req, &dot_a);
    const bool inpl_b = perm_b && inplace_dot(b_src, b_labels, b_req, &dot_b);
    if (perm_a && !inpl_a && !(gather && !small_is_a)) {
      build_perm_desc(a_labels.data(), (int)a_labels.size(), a_req.data(), (int)a_req.size(), slice_labels.data(),
                      ns, PM_C64, nK, &d);
      TNQ_CUDA(perm(ctx, d, a_src, scratch_a, nullptr, slice_id, 16.0 * std::ldexp(1.0, (int)a_req.size())));
    }
    if (perm_b && !inpl_b && !(gather && small_is_a)) {
      build_perm_desc(b_labels.data(), (int)b_labels.size(), b_req.data(), (int)b_req.size(), slice_labels.data(),
                      ns, PM_C64, nK, &d);
      TNQ_CUDA(perm(ctx, d, b_src, scratch_b, nullptr, slice_id, 16.0 * std::ldexp(1.0, (int)b_req.size())));
    }
    if (gather) {
      // large operand: required order [K][rows][H]; find each bit in its stored labels
      const std::vector<int>& src_l = small_is_a ? b_labels : a_labels;
      const std::vector<int>& req = small_is_a ? b_req : a_req;
      auto spos = [&](int l) { return int(std::find(src_l.begin(), src_l.end(), l) - src_l.begin()); };
      GatherDesc gd;
      gd.nk = nK;
      for (int j = 0; j < nK; ++j) gd.kpos[j] = spos(req[j]);
      gd.nrow = (int)req.size() - nK;
      for (int j = 0; j < gd.nrow; ++j) gd.rowpos[j] = spos(req[nK + j]);
      gd.n_slice = ns;
      for (int j = 0; j < 32; ++j) gd.slice_src[j] = j < ns ? spos(slice_labels[j]) : -1;
      for (int j = 0; j < ns; ++j)
        if (gd.slice_src[j] >= (int)src_l.size()) gd.slice_src[j] = -1;
      const int M = 1 << nM, N = 1 << nN, K = 1 << nK, H = 1 << nH;
      const void* Ssm = small_is_a ? (perm_a ? (const void*)scratch_a : a_src) : (perm_b ? (const void*)scratch_b : b_src);
      const void* Gs = small_is_a ? b_src : a_src;
      KernelRecord r{4, ctx->cur_step, nH, nM, nN, nK, 8.0 * work,
                     8.0 * (std::ldexp(1.0, nH + nM + nK) + std::ldexp(1.0, nH + nN + nK) +
                            (acc ? 2.0 : 1.0) * std::ldexp(1.0, nH + nM + nN)),
                     0.f};
      if (tc_rows_ok) r.kind = 5;
      int slot = timing_begin(ctx);
      cudaError_t e;
      if (tc_rows_ok)
        e = small_is_a ? launch_cgemm_tc_rows(Ssm, Gs, gd, C, acc, M, N, K, H, N, 1, slice_id, ctx->precision, err,
                                              ctx->sm_count, ctx->stream, tr_scratch, tr_avail)
                       : launch_cgemm_tc_rows(Ssm, Gs, gd, C, acc, N, M, K, H, 1, N, slice_id, ctx->precision, err,
                                              ctx->sm_count, ctx->stream, tr_scratch, tr_avail);
      else
        e = small_is_a ? launch_cgemm_rows_gather(Ssm, Gs, gd, C, acc, M, N, K, H, N, 1, slice_id, ctx->stream)
                       : launch_cgemm_rows_gather(Ssm, Gs, gd, C, acc, N, M, K, H, 1, N, slice_id, ctx->stream);
      timing_end(ctx, slot, r);
      TNQ_CUDA(e);
      ctx->launches++;
      return TNQ_OK;
    }
    const void* A = perm_a ? (const void*)scratch_a : a_src;
    const void* B = perm_b ? (const void*)scratch_b : b_src;
    const int M = 1 << nM, N = 1 << nN, K = 1 << nK, H = 1 << nH;
    KernelRecord r{4, ctx->cur_step, nH, nM, nN, nK, 8.0 * work,
                   8.0 * (std::ldexp(1.0, nH + nM + nK) + std::ldexp(1.0, nH + nN + nK) +
                          (acc ? 2.0 : 1.0) * std::ldexp(1.0, nH + nM + nN)),
                   0.f};
    int slot = timing_begin(ctx);
    cudaError_t e;
    int splits;
    if (use_dot(nM, nN, nK)) {
      splits = dot_splits(nH, nM, nN, nK);
      if (!inpl_a) dot_a = dot_contiguous(A, M, K, H);
      if (!inpl_b) dot_b = dot_contiguous(B, N, K, H);
      e = launch_cdot_ops(dot_a, dot_b, part, splits, M, N, K, H, ctx->stream);
      if (e == cudaSuccess) e = launch_reduce_splits(part, splits, out_elems, C, acc, ctx->sm_count, ctx->stream);
    } else {
      splits = rows_splits(nH, nM, nN, nK);
      if (nM <= nN)
        e = launch_cgemm_rows(A, B, C, acc, part, splits, M, N, K, H, N, 1, ctx->stream);
      else
        e = launch_cgemm_rows(B, A, C, acc, part, splits, N, M, K, H, 1, N, ctx->stream);
      if (e == cudaSuccess && splits > 1)
        e = launch_reduce_splits(part, splits, out_elems, C, acc, ctx->sm_count, ctx->stream);
    }
    timing_end(ctx, slot, r);
    TNQ_CUDA(e);
    ctx->launches += (use_dot(nM, nN, nK) || splits > 1) ? 2 : 1;
    return TNQ_OK;
  }
  if (prec == TNQ_PREC_FP32) {
    if (perm_a) {
      build_perm_desc(a_labels.data(), (int)a_labels.size(), a_req.data(), (int)a_req.size(), slice_labels.data(),
                      ns, PM_C64, nK, &d);
      TNQ_CUDA(perm(ctx, d, a_src, scratch_a, nullptr, slice_id, 16.0 * std::ldexp(1.0, (int)a_req.size())));
      op.a0 = scratch_a;
    } else {
      op.a0 = a_src;
    }
    if (perm_b) {
      build_perm_desc(b_labels.data(), (int)b_labels.size(), b_req.data(), (int)b_req.size(), slice_labels.data(),
                      ns, PM_C64, nK, &d);
      TNQ_CUDA(perm(ctx, d, b_src, scratch_b, nullptr, slice_id, 16.0 * std::ldexp(1.0, (int)b_req.size())));
      op.b0 = scratch_b;
    } else {
      op.b0 = b_src;
    }
    KernelRecord r{1, ctx->cur_step, nH, nM, nN, nK, 8.0 * work,
                   8.0 * (std::ldexp(1.0, nH + nM + nK) + std::ldexp(1.0, nH + nN + nK) +
                          (acc ? 2.0 : 1.0) * std::ldexp(1.0, nH + nM + nN)),
                   0.f};
    const int splits = part ? simt_splits(nH, nM, nN, nK) : 1;
    int slot = timing_begin(ctx);
    TNQ_CUDA(launch_cgemm_simt(op.a0, op.b0, C, acc, part, splits, 1 << nM, 1 << nN, 1 << nK, 1 << nH, ctx->stream));
    if (splits > 1) {
      TNQ_CUDA(launch_reduce_splits(part, splits, out_elems, C, acc, ctx->sm_count, ctx->stream));
      ctx->launches++;
    }
    timing_end(ctx, slot, r);
    ctx->launches++;
    return TNQ_OK;
  }
  // tensor-core modes: A is always expanded (and split), B split unless plain TF32 in place
  size_t na = size_t(1) << a_req.size(), nb = size_t(1) << b_req.size();
  build_perm_desc(a_labels.data(), (int)a_labels.size(), a_req.data(), (int)a_req.size(), slice_labels.data(), ns,
                  tc_mode_a(prec), nK, &d);
  char* a1 = scratch_a + ((a_half_bytes(prec, na) + 1023) & ~size_t(1023));
  TNQ_CUDA(perm(ctx, d, a_src, scratch_a, a1, slice_id, 8.0 * na + a_half_bytes(prec, na) * (prec == TNQ_PREC_TF32 ? 1 : 2)));
  op.a0 = scratch_a;
  op.a1 = prec == TNQ_PREC_TF32 ? nullptr : a1;
  if (prec == TNQ_PREC_TF32 && !perm_b) {
    op.b0 = b_src;
  } else {
    build_perm_desc(b_labels.data(), (int)b_labels.size(), b_req.data(), (int)b_req.size(), slice_labels.data(),
                    ns, tc_mode_b(prec), nK, &d);
    char* b1 = scratch_b + ((b_half_bytes(prec, nb) + 1023) & ~size_t(1023));
    TNQ_CUDA(perm(ctx, d, b_src, scratch_b, b1, slice_id, 8.0 * nb + b_half_bytes(prec, nb) * (prec == TNQ_PREC_TF32 ? 1 : 2)));
    op.b0 = scratch_b;
    op.b1 = prec == TNQ_PREC_TF32 ? nullptr : b1;
  }
  TcGemmArgs g;
  g.a_hi = op.a0;
  g.a_lo = op.a1;
  g.b_hi = op.b0;
  g.b_lo = op.b1;
  g.c = C;
  g.acc = acc;
  g.M = 1 << nM;
  g.N = 1 << nN;
  g.K = 1 << nK;
  g.batch = 1 << nH;
  g.precision = prec;
  g.err = err;
  int used = 1;
  g.splits = part ? tc_splits(nH, nM, nN, nK, prec == TNQ_PREC_BF16X3) : 1;
  g.part = part;
  g.splits_used = &used;
  const double op_bytes = prec == TNQ_PREC_BF16X3 ? 2.0 : 4.0;
  const double npass = prec == TNQ_PREC_TF32 ? 1.0 : 2.0;
  KernelRecord r{2, ctx->cur_step, nH, nM, nN, nK, 8.0 * work,
                 npass * op_bytes * (4.0 * std::ldexp(1.0, nH + nM + nK) + 2.0 * std::ldexp(1.0, nH + nN + nK)) +
                     (acc ? 16.0 : 8.0) * std::ldexp(1.0, nH + nM + nN),
                 0.f};
  int slot = timing_begin(ctx);
  cudaError_t e = launch_cgemm_tc(g, ctx->sm_count, ctx->stream);
  if (e == cudaSuccess && used > 1) {
    e = launch_reduce_splits(part, used, out_elems, C, acc, ctx->sm_count, ctx->stream);
    ctx->launches++;
  }
  timing_end(ctx, slot, r);
  if (e == cudaErrorNotSupported)
    return fail(TNQ_ERR_NOT_SUPPORTED, "tensor-core GEMM unavailable for this shape/precision");
  TNQ_CUDA(e);
  ctx->launches++;
  return TNQ_OK;
}

tnq_status run_step(Ctx* ctx, Plan* p, size_t si, int slice_id, char* ws, int choice) {
  static const std::vector<int> kNoSlices;
  auto& s = p->steps[si];
  auto& ta = p->tensors[s.a];
  auto& tb = p->tensors[s.b];
  void* acc = s.out == p->root ? (void*)(ws + p->ws_acc) : nullptr;
  void* C = s.out == p->root ? nullptr : (void*)(ws + p->tensors[s.out].offset);
  // a slice-batched step keeps the sliced indices: nothing is fixed to a slice
  const std::vector<int>& sl = s.sliced_batch ? kNoSlices : p->slice_labels;
  return run_gemm_step(ctx, ws + ta.offset, ta.labels, s.perm_a, ws + tb.offset, tb.labels, s.perm_b, s.a_req,
                       s.b_req, sl, s.sliced_batch ? 0 : slice_id, s.nH, s.nM, s.nN, s.nK, ws + p->ws_scratch_a,
                       ws + p->ws_scratch_b, C, acc, reinterpret_cast<int*>(ws + p->ws_misc + 4),
                       ws + p->ws_partial, p->ws_scratch_b - p->ws_scratch_a, choice);
}

// Kernel choice of a step under TNQ_KERNELS_TENSOR_CORES: the tall-skinny
// tensor-core kernel where the shape qualifies, else the general tensor-core
// GEMM where it is supported, else the default rule.
int forced_tc_choice(const Ctx* ctx, const Step& s) {
  if (ctx->precision == TNQ_PREC_FP32) return -1;
  const int n_small = std::min(s.nM, s.nN), n_big = std::max(s.nM, s.nN);
  if (n_small <= 7 && !use_dot(s.nM, s.nN, s.nK) &&
      tc_rows_supported(1 << n_small, 1 << n_big, 1 << s.nK, 1 << s.nH, n_big + s.nH, ctx->precision))
    return 2;
  if (tc_gemm_supported(1 << s.nM, 1 << s.nN, 1 << s.nK, ctx->precision)) return 1;
  return -1;
}

// One slice of a batch; slice-invariant steps run only in the batch's first
// slice (their outputs persist for the batch).
tnq_status run_pass(Ctx* ctx, Plan* p, int slice_id, char* ws, bool first) {
  const bool tuned = p->tuned_precision == ctx->precision && p->kernel_choice.size() == p->steps.size();
  const bool forced = ctx->kernel_policy == TNQ_KERNELS_TENSOR_CORES;
  for (size_t si = 0; si < p->steps.size(); ++si) {
    if (p->steps[si].fold) continue;  // contracted when the plan was bound
    if (p->steps[si].once() && !first) continue;
    ctx->cur_step = (int)si;
    const int choice = forced ? forced_tc_choice(ctx, p->steps[si]) : tuned ? p->kernel_choice[si] : -1;
    tnq_status st = run_step(ctx, p, si, slice_id, ws, choice);
    if (st != TNQ_OK) return st;
  }
  ctx->cur_step = -1;
  return TNQ_OK;
}


// Contract the plan's constant subtrees (steps whose leaves are all static)
// once for the context's precision; their outputs persist in the workspace.
tnq_status ensure_folded(Ctx* ctx, Plan* p) {
  if (p->folded_precision == ctx->precision) return TNQ_OK;
  char* ws = static_cast<char*>(p->bound_ws);
  const bool tuned = p->tuned_precision == ctx->precision && p->kernel_choice.size() == p->steps.size();
  const bool forced = ctx->kernel_policy == TNQ_KERNELS_TENSOR_CORES;
  for (size_t si = 0; si < p->steps.size(); ++si) {
    if (!p->steps[si].fold) continue;
    ctx->cur_step = (int)si;
    const int choice = forced ? forced_tc_choice(ctx, p->steps[si]) : tuned ? p->kernel_choice[si] : -1;
    tnq_status st = run_step(ctx, p, si, 0, ws, choice);
    if (st != TNQ_OK) return st;
  }
  ctx->cur_step = -1;
  p->folded_precision = ctx->precision;
  return TNQ_OK;
}

}  // namespace

void plan_release_graph(Plan* p) {
  if (p->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(p->graph_exec));
  p->graph_exec = nullptr;
  p->graph_precision = -1;
  p->graph_policy = -1;
}

namespace {

// Enqueue one full batch that reads its bitstrings from the staging buffer and
// leaves its amplitudes (bitstring order) in the output staging buffer.
tnq_status enqueue_batch(Ctx* ctx, Plan* p, int64_t nv) {
  char* ws = static_cast<char*>(p->bound_ws);
  const int w = p->batch_log2;
  std::vector<int> bpos, opos;
  root_positions(p, &bpos, &opos);
  TNQ_CUDA(fill_projections(ctx, proj_leaves(p, ws), w, reinterpret_cast<const int8_t*>(ws + p->ws_bits), nv,
                            reinterpret_cast<int*>(ws + p->ws_misc)));
  TNQ_CUDA(launch_zero(ws + p->ws_acc, 16 * (size_t(1) << p->tensors[p->root].rank), ctx->stream));
  const int n_slices = 1 << p->slice_labels.size();
  for (int s = 0; s < n_slices; ++s) {
    tnq_status st = run_pass(ctx, p, s, ws, s == 0);
    if (st != TNQ_OK) return st;
  }
  TNQ_CUDA(launch_finalize(ws + p->ws_acc, ws + p->ws_out_stage, nv, bpos.data(), w, opos.data(), (int)opos.size(),
                           p->density, ctx->stream));
  ctx->launches++;
  return TNQ_OK;
}

// Capture enqueue_batch for a full batch into a graph (once per plan and precision).
tnq_status ensure_graph(Ctx* ctx, Plan* p) {
  if (p->graph_exec && p->graph_precision == ctx->precision && p->graph_policy == ctx->kernel_policy) return TNQ_OK;
  plan_release_graph(p);
  auto t0 = std::chrono::steady_clock::now();
  if (ctx->precision != TNQ_PREC_FP32) TNQ_CUDA(tc_gemm_prepare());
  // capture on a private stream (the legacy default stream cannot be captured);
  // the graph is launched on the context's stream
  if (!ctx->capture_stream) TNQ_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  const uint64_t launches_before = ctx->launches;
  cudaStream_t user_stream = ctx->stream;
  ctx->stream = ctx->capture_stream;
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    ctx->stream = user_stream;
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  tnq_status st = enqueue_batch(ctx, p, int64_t(1) << p->batch_log2);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->stream = user_stream;
  ctx->launches = launches_before;  // captured, not launched
  if (st != TNQ_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  p->graph_exec = ex;
  p->graph_precision = ctx->precision;
  p->graph_policy = ctx->kernel_policy;
  p->graph_nodes = (int64_t)nodes;
  p->graph_capture_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return TNQ_OK;
}

}  // namespace

tnq_status exec_bind(Ctx* ctx, Plan* p, void* ws, size_t bytes) {
  if (!ws) return fail(TNQ_ERR_WORKSPACE, "workspace is NULL");
  if (bytes < p->ws_total)
    return fail(TNQ_ERR_WORKSPACE, "workspace too small: need " + std::to_string(p->ws_total) + " bytes");
  if (!is_device_ptr(ws)) return fail(TNQ_ERR_WORKSPACE, "workspace must be device memory");
  TNQ_CUDA(cudaSetDevice(ctx->device));
  plan_release_graph(p);
  char* base = static_cast<char*>(ws);
  std::vector<float> buf;
  for (size_t i = 0; i < p->net.leaves.size(); ++i) {
    const Leaf& L = p->net.leaves[i];
    if (L.kind != LEAF_STATIC) continue;
    buf.resize(2 * L.data.size());
    for (size_t k = 0; k < L.data.size(); ++k) {
      buf[2 * k] = (float)L.data[k].real();
      buf[2 * k + 1] = (float)L.data[k].imag();
    }
    TNQ_CUDA(cudaMemcpyAsync(base + p->tensors[i].offset, buf.data(), buf.size() * sizeof(float),
                             cudaMemcpyHostToDevice, ctx->stream));
    TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  if (!p->traj_leaves.empty()) {
    std::vector<double> mats(2 * p->traj_mats.size());
    for (size_t k = 0; k < p->traj_mats.size(); ++k) {
      mats[2 * k] = p->traj_mats[k].real();
      mats[2 * k + 1] = p->traj_mats[k].imag();
    }
    TNQ_CUDA(cudaMemcpyAsync(base + p->ws_traj, p->traj_leaves.data(), sizeof(TrajLeafDesc) * p->traj_leaves.size(),
                             cudaMemcpyHostToDevice, ctx->stream));
    TNQ_CUDA(cudaMemcpyAsync(base + p->ws_traj_factors, p->traj_factors.data(),
                             sizeof(TrajFactor) * p->traj_factors.size(), cudaMemcpyHostToDevice, ctx->stream));
    TNQ_CUDA(cudaMemcpyAsync(base + p->ws_traj_mats, mats.data(), 8 * mats.size(), cudaMemcpyHostToDevice,
                             ctx->stream));
    if (!p->traj_cumq.empty())
      TNQ_CUDA(cudaMemcpyAsync(base + p->ws_traj_cumq, p->traj_cumq.data(), 8 * p->traj_cumq.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
    TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  if (!p->picks.empty()) {
    TNQ_CUDA(cudaMemcpyAsync(base + p->ws_picks, p->picks.data(), p->picks.size(), cudaMemcpyHostToDevice,
                             ctx->stream));
    TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  {
    std::vector<int> tab = p->net.proj_src;
    tab.insert(tab.end(), p->net.open_qubits.begin(), p->net.open_qubits.end());
    if (!tab.empty()) {
      TNQ_CUDA(cudaMemcpyAsync(base + p->ws_qtab, tab.data(), 4 * tab.size(), cudaMemcpyHostToDevice, ctx->stream));
      TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
  }
  p->bound_ws = ws;
  p->bound_bytes = bytes;
  p->folded_precision = -1;
  return TNQ_OK;
}

tnq_status exec_amplitudes(Ctx* ctx, Plan* p, int64_t n_bs, const int8_t* bits, double* out) {
  return exec_amplitudes_range(ctx, p, n_bs, bits, 0, int64_t(1) << p->slice_labels.size(), out);
}

tnq_status exec_amplitudes_range(Ctx* ctx, Plan* p, int64_t n_bs, const int8_t* bits, int64_t slice_begin,
                                 int64_t slice_count, double* out) {
  if (!p->bound_ws) return fail(TNQ_ERR_WORKSPACE, "plan has no bound workspace");
  if (p->expectation) return fail(TNQ_ERR_INVALID_ARG, "expectation-value plan; use tnq_expectation");
  if (p->net.noisy) return fail(TNQ_ERR_INVALID_ARG, "plan is for a noisy circuit; use tnq_noisy_probabilities");
  if (n_bs < 0 || (n_bs > 0 && (!bits || !out))) return fail(TNQ_ERR_INVALID_ARG, "bad bitstring/output buffers");
  if (n_bs == 0) return TNQ_OK;
  TNQ_CUDA(cudaSetDevice(ctx->device));
  char* ws = static_cast<char*>(p->bound_ws);
  const int rl = p->net.row_len, w = p->batch_log2;
  const int64_t per = int64_t(1) << w;
  const int64_t n_out = int64_t(1) << p->net.open_qubits.size();  // amplitudes per bitstring
  const int64_t vals = p->density ? 1 : 2;                          // doubles per result
  const bool bits_dev = is_device_ptr(bits), out_dev = is_device_ptr(out);
  if (!bits_dev && !host_bits_ok(p, n_bs, bits))
    return fail(TNQ_ERR_INVALID_ARG, p->net.open_qubits.empty()
                                         ? "bitstring entries must be 0 or 1"
                                         : "bitstring entries must be -1 at the plan's open qubits and 0 or 1 elsewhere");
  int* err_flag = reinterpret_cast<int*>(ws + p->ws_misc);
  int8_t* bits_stage = reinterpret_cast<int8_t*>(ws + p->ws_bits);
  double* out_stage = reinterpret_cast<double*>(ws + p->ws_out_stage);
  const ProjLeaves pl = proj_leaves(p, ws);
  std::vector<int> bpos, opos;
  root_positions(p, &bpos, &opos);
  TNQ_CUDA(cudaMemsetAsync(err_flag, 0, 2 * sizeof(int), ctx->stream));
  const size_t acc_bytes = 16 * (size_t(1) << p->tensors[p->root].rank);
  const int64_t n_slices = int64_t(1) << p->slice_labels.size();
  if (slice_begin < 0 || slice_count < 0 || slice_begin + slice_count > n_slices)
    return fail(TNQ_ERR_INVALID_ARG, "slice range outside [0, 2^n_sliced)");
  // the captured graph covers every slice; partial ranges launch directly
  const bool graphs = ctx->use_graphs && !ctx->timing && slice_begin == 0 && slice_count == n_slices;
  {
    tnq_status st = ensure_folded(ctx, p);
    if (st != TNQ_OK) return st;
  }
  for (int64_t base = 0; base < n_bs; base += per) {
    int64_t nv = std::min<int64_t>(per, n_bs - base);
    const size_t out_bytes = size_t(nv * n_out * vals) * 8;
    if (graphs && nv == per) {
      // full batch: stage the bitstrings, replay the captured graph, copy out
      TNQ_CUDA(cudaMemcpyAsync(bits_stage, bits + base * rl, size_t(nv) * rl,
                               bits_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
      tnq_status st = ensure_graph(ctx, p);
      if (st != TNQ_OK) return st;
      TNQ_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(p->graph_exec), ctx->stream));
      ctx->launches += uint64_t(p->graph_nodes);
      TNQ_CUDA(cudaMemcpyAsync(out + vals * base * n_out, out_stage, out_bytes,
                               out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
      continue;
    }
    const int8_t* bsrc;
    if (bits_dev) {
      bsrc = bits + base * rl;
    } else {
      TNQ_CUDA(cudaMemcpyAsync(bits_stage, bits + base * rl, size_t(nv) * rl, cudaMemcpyHostToDevice, ctx->stream));
      bsrc = bits_stage;
    }
    TNQ_CUDA(fill_projections(ctx, pl, w, bsrc, nv, err_flag));
    TNQ_CUDA(launch_zero(ws + p->ws_acc, acc_bytes, ctx->stream));
    for (int64_t s = slice_begin; s < slice_begin + slice_count; ++s) {
      tnq_status st = run_pass(ctx, p, int(s), ws, s == slice_begin);
      if (st != TNQ_OK) return st;
    }
    double* dst = out_dev ? out + vals * base * n_out : out_stage;
    TNQ_CUDA(launch_finalize(ws + p->ws_acc, dst, nv, bpos.data(), w, opos.data(), (int)opos.size(), p->density,
                             ctx->stream));
    ctx->launches++;
    if (!out_dev)
      TNQ_CUDA(cudaMemcpyAsync(out + vals * base * n_out, out_stage, out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
  }
  int herr[2] = {0, 0};
  TNQ_CUDA(cudaMemcpyAsync(herr, err_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->timing) {
    tnq_status ts = timing_collect(ctx);
    if (ts != TNQ_OK) return ts;
  }
  if (herr[1]) return fail(TNQ_ERR_TIMEOUT, "a tensor-core GEMM wait expired; results are invalid");
  if (herr[0])
    return fail(TNQ_ERR_INVALID_ARG, p->net.open_qubits.empty()
                                         ? "bitstring entries must be 0 or 1"
                                         : "bitstring entries must be -1 at the plan's open qubits and 0 or 1 elsewhere");
  return TNQ_OK;
}

tnq_status exec_autotune(Ctx* ctx, Plan* p, int reps, int* n_tc, int* n_cuda) {
  if (!p->bound_ws) return fail(TNQ_ERR_WORKSPACE, "plan has no bound workspace");
  TNQ_CUDA(cudaSetDevice(ctx->device));
  if (ctx->precision != TNQ_PREC_FP32) TNQ_CUDA(tc_gemm_prepare());
  char* ws = static_cast<char*>(p->bound_ws);
  const size_t n = p->steps.size();
  std::vector<int8_t> choice(n, -1);
  cudaEvent_t e0, e1;
  TNQ_CUDA(cudaEventCreate(&e0));
  TNQ_CUDA(cudaEventCreate(&e1));
  const bool timing = ctx->timing;
  ctx->timing = false;
  int ntc = 0, ncc = 0;
  tnq_status result = TNQ_OK;
  for (size_t si = 0; si < n && result == TNQ_OK; ++si) {
    const Step& s = p->steps[si];
    const bool tc_ok = ctx->precision != TNQ_PREC_FP32 &&
                       tc_gemm_supported(1 << s.nM, 1 << s.nN, 1 << s.nK, ctx->precision) &&
                       s.nM + s.nN + s.nK + s.nH >= 12;
    // candidates: 0 CUDA cores, 1 tensor-core GEMM, 2 tall-skinny tensor-core kernel
    const int n_small = std::min(s.nM, s.nN), n_big = std::max(s.nM, s.nN);
    const bool rows_ok = ctx->precision != TNQ_PREC_FP32 && n_small <= 7 && !use_dot(s.nM, s.nN, s.nK) &&
                         s.nM + s.nN + s.nK + s.nH >= 12 &&
                         tc_rows_supported(1 << n_small, 1 << n_big, 1 << s.nK, 1 << s.nH, n_big + s.nH,
                                           ctx->precision);
    int cands[3], nc = 0;
    cands[nc++] = 0;
    if (tc_ok) cands[nc++] = 1;
    if (rows_ok) cands[nc++] = 2;
    if (nc == 1) continue;  // one candidate only
    float best = 0;
    int pick = -1;
    for (int ci = 0; ci < nc && result == TNQ_OK; ++ci) {
      const int c = cands[ci];
      float tmin = 1e30f;
      for (int r = 0; r < reps + 1; ++r) {  // first run warms up
        cudaEventRecord(e0, ctx->stream);
        result = run_step(ctx, p, si, 0, ws, c);
        cudaEventRecord(e1, ctx->stream);
        if (result != TNQ_OK) break;
        cudaError_t er = cudaEventSynchronize(e1);
        if (er != cudaSuccess) {
          result = cuda_fail(er, "autotune");
          break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) tmin = std::min(tmin, ms);
      }
      if (pick < 0 || tmin < best) {
        pick = c;
        best = tmin;
      }
    }
    choice[si] = (int8_t)pick;
    (pick >= 1 ? ntc : ncc)++;
  }
  ctx->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != TNQ_OK) return result;
  int herr = 0;
  TNQ_CUDA(cudaMemcpy(&herr, ws + p->ws_misc + 4, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return fail(TNQ_ERR_TIMEOUT, "a tensor-core GEMM wait expired during autotuning");
  p->kernel_choice = choice;
  p->tuned_precision = ctx->precision;
  p->folded_precision = -1;  // the timing runs overwrote the folded outputs
  plan_release_graph(p);
  if (n_tc) *n_tc = ntc;
  if (n_cuda) *n_cuda = ncc;
  return TNQ_OK;
}

namespace {

// SplitMix64 (Steele, Lea & Flood 2014) on the host: the uniform in [0, 1)
// of trajectory t, channel c, the same draw the trajectory kernel makes.
double host_uniform(uint64_t seed, uint64_t traj, uint64_t chan) {
  const uint64_t i = (traj << 32) + chan + 1;
  uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return double(z >> 11) * (1.0 / 9007199254740992.0);
}

// Distinct trajectories among 0 .. n_traj - 1: every channel's pick drawn as
// on the device, equal pick vectors grouped (in order of first appearance)
// with their multiplicities.  The mean of |amp|^2 over all trajectories is the
// multiplicity-weighted mean over the distinct ones, exactly.
void distinct_trajectories(const Plan* p, uint64_t seed, int64_t n_traj, std::vector<int8_t>* picks,
                           std::vector<double>* mult) {
  const size_t nch = p->chan_cumq.size();
  std::map<std::vector<int8_t>, size_t> index;
  std::vector<int8_t> v(nch);
  picks->clear();
  mult->clear();
  for (int64_t t = 0; t < n_traj; ++t) {
    for (size_t c = 0; c < nch; ++c) {
      const auto& cq = p->chan_cumq[c];
      const double u = host_uniform(seed, uint64_t(t), uint64_t(c));
      int k = (int)cq.size() - 1;
      for (int j = 0; j < (int)cq.size(); ++j)
        if (u < cq[j]) {
          k = j;
          break;
        }
      v[c] = int8_t(k);
    }
    auto it = index.find(v);
    if (it == index.end()) {
      index.emplace(v, mult->size());
      picks->insert(picks->end(), v.begin(), v.end());
      mult->push_back(1.0);
    } else {
      (*mult)[it->second] += 1.0;
    }
  }
}

// Shared driver of the noisy calls: for every batch of bitstrings and every
// chunk of 2^traj_log2 trajectories, build the trajectory leaves, contract all
// slices into the FP64 accumulator, then hand the accumulator to `consume`.
// With `distinct` (host picks [n_units][n_channels] and multiplicities) the
// chunks run over those distinct trajectories instead of drawing on the GPU.
template <typename Consume, typename BatchEnd>
tnq_status noisy_driver(Ctx* ctx, Plan* p, int64_t traj_begin, int64_t n_traj, uint64_t seed, int64_t n_bs,
                        const int8_t* bits, Consume consume, BatchEnd batch_end,
                        const std::vector<int8_t>* distinct = nullptr, const std::vector<double>* mult = nullptr) {
  char* ws = static_cast<char*>(p->bound_ws);
  const int n = p->net.row_len, w = p->batch_log2, t = p->traj_log2;
  const int64_t per = int64_t(1) << w, tper = int64_t(1) << t;
  const bool bits_dev = is_device_ptr(bits);
  if (!bits_dev && !host_bits_ok(p, n_bs, bits))
    return fail(TNQ_ERR_INVALID_ARG, "bitstring entries must be 0 or 1");
  int* err_flag = reinterpret_cast<int*>(ws + p->ws_misc);
  int8_t* bits_stage = reinterpret_cast<int8_t*>(ws + p->ws_bits);
  const ProjLeaves pl = proj_leaves(p, ws);
  const auto& rl = p->tensors[p->root].labels;
  std::vector<int> bpos(w), tpos(t);
  for (int j = 0; j < w; ++j) bpos[j] = int(std::find(rl.begin(), rl.end(), p->net.batch_labels[j]) - rl.begin());
  for (int j = 0; j < t; ++j) tpos[j] = int(std::find(rl.begin(), rl.end(), p->net.traj_labels[j]) - rl.begin());
  TNQ_CUDA(cudaMemsetAsync(err_flag, 0, 2 * sizeof(int), ctx->stream));
  const size_t acc_bytes = 16 * (size_t(1) << p->tensors[p->root].rank);
  const int n_slices = 1 << p->slice_labels.size();
  {
    tnq_status st = ensure_folded(ctx, p);
    if (st != TNQ_OK) return st;
  }
  for (int64_t base = 0; base < n_bs; base += per) {
    const int64_t nv = std::min<int64_t>(per, n_bs - base);
    const int8_t* bsrc;
    if (bits_dev) {
      bsrc = bits + base * n;
    } else {
      TNQ_CUDA(cudaMemcpyAsync(bits_stage, bits + base * n, size_t(nv) * n, cudaMemcpyHostToDevice, ctx->stream));
      bsrc = bits_stage;
    }
    TNQ_CUDA(fill_projections(ctx, pl, w, bsrc, nv, err_flag));
    tnq_status st = consume(-1, base, nv, 0, 0, bpos, tpos);  // batch start
    if (st != TNQ_OK) return st;
    const int64_t units = distinct ? int64_t(mult->size()) : n_traj;
    const size_t nch = p->chan_cumq.size();
    for (int64_t tb = 0; tb < units; tb += tper) {
      const int64_t nt = std::min<int64_t>(tper, units - tb);
      if (distinct) {
        TNQ_CUDA(cudaMemcpyAsync(ws + p->ws_dedup_picks, distinct->data() + size_t(tb) * nch, size_t(nt) * nch,
                                 cudaMemcpyHostToDevice, ctx->stream));
        TNQ_CUDA(cudaMemcpyAsync(ws + p->ws_dedup_w, mult->data() + tb, size_t(nt) * 8, cudaMemcpyHostToDevice,
                                 ctx->stream));
        TNQ_CUDA(launch_traj_leaves(reinterpret_cast<const TrajLeafDesc*>(ws + p->ws_traj),
                                    (int)p->traj_leaves.size(),
                                    reinterpret_cast<const TrajFactor*>(ws + p->ws_traj_factors),
                                    reinterpret_cast<const double2*>(ws + p->ws_traj_mats),
                                    reinterpret_cast<const double*>(ws + p->ws_traj_cumq), ws, seed, 0, t, ctx->stream,
                                    reinterpret_cast<const int8_t*>(ws + p->ws_dedup_picks), int(nch), nt));
      } else {
        TNQ_CUDA(launch_traj_leaves(reinterpret_cast<const TrajLeafDesc*>(ws + p->ws_traj),
                                    (int)p->traj_leaves.size(),
                                    reinterpret_cast<const TrajFactor*>(ws + p->ws_traj_factors),
                                    reinterpret_cast<const double2*>(ws + p->ws_traj_mats),
                                    reinterpret_cast<const double*>(ws + p->ws_traj_cumq), ws, seed,
                                    uint64_t(traj_begin + tb), t, ctx->stream));
      }
      ctx->launches++;
      TNQ_CUDA(launch_zero(ws + p->ws_acc, acc_bytes, ctx->stream));
      for (int s = 0; s < n_slices; ++s) {
        st = run_pass(ctx, p, s, ws, s == 0);
        if (st != TNQ_OK) return st;
      }
      st = consume(0, base, nv, tb, nt, bpos, tpos);
      if (st != TNQ_OK) return st;
    }
    st = batch_end(base, nv);
    if (st != TNQ_OK) return st;
  }
  int herr[2] = {0, 0};
  TNQ_CUDA(cudaMemcpyAsync(herr, err_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->timing) {
    tnq_status ts = timing_collect(ctx);
    if (ts != TNQ_OK) return ts;
  }
  if (herr[1]) return fail(TNQ_ERR_TIMEOUT, "a tensor-core GEMM wait expired; results are invalid");
  if (herr[0]) return fail(TNQ_ERR_INVALID_ARG, "bitstring entries must be 0 or 1");
  return TNQ_OK;
}

tnq_status noisy_checks(Plan* p, int64_t n_traj, int64_t n_bs, const int8_t* bits, const void* out) {
  if (!p->bound_ws) return fail(TNQ_ERR_WORKSPACE, "plan has no bound workspace");
  if (!p->net.noisy || p->expectation) return fail(TNQ_ERR_INVALID_ARG, "plan is for a circuit without channels");
  if (!p->net.open_qubits.empty()) return fail(TNQ_ERR_NOT_SUPPORTED, "noisy plans with open qubits");
  if (n_traj < 1) return fail(TNQ_ERR_INVALID_ARG, "n_traj must be >= 1");
  if (n_bs < 0 || (n_bs > 0 && (!bits || !out))) return fail(TNQ_ERR_INVALID_ARG, "bad bitstring/output buffers");
  return TNQ_OK;
}

}  // namespace

tnq_status exec_noisy(Ctx* ctx, Plan* p, int64_t n_traj, uint64_t seed, int64_t n_bs, const int8_t* bits,
                      double* p_out, double* se_out) {
  tnq_status st = noisy_checks(p, n_traj, n_bs, bits, p_out);
  if (st != TNQ_OK || n_bs == 0) return st;
  TNQ_CUDA(cudaSetDevice(ctx->device));
  char* ws = static_cast<char*>(p->bound_ws);
  double* psum = reinterpret_cast<double*>(ws + p->ws_psum);
  double* p2sum = reinterpret_cast<double*>(ws + p->ws_p2sum);
  double* stage = reinterpret_cast<double*>(ws + p->ws_out_stage);
  const int64_t per = int64_t(1) << p->batch_log2;
  const bool p_dev = is_device_ptr(p_out), se_dev = se_out && is_device_ptr(se_out);
  auto consume = [&](int phase, int64_t, int64_t nv, int64_t, int64_t nt, const std::vector<int>& bpos,
                     const std::vector<int>& tpos) -> tnq_status {
    if (phase < 0) {
      TNQ_CUDA(cudaMemsetAsync(psum, 0, 8 * per, ctx->stream));
      TNQ_CUDA(cudaMemsetAsync(p2sum, 0, 8 * per, ctx->stream));
      return TNQ_OK;
    }
    TNQ_CUDA(launch_noisy_accumulate(ws + p->ws_acc, nv, nt, bpos.data(), (int)bpos.size(), tpos.data(),
                                     (int)tpos.size(), psum, p2sum, ctx->stream,
                                     reinterpret_cast<const double*>(ws + p->ws_dedup_w)));
    ctx->launches++;
    return TNQ_OK;
  };
  auto batch_end = [&](int64_t base, int64_t nv) -> tnq_status {
    double* pd = p_dev ? p_out + base : stage;
    double* sd = se_out ? (se_dev ? se_out + base : stage + per) : nullptr;
    TNQ_CUDA(launch_noisy_finalize(psum, p2sum, nv, n_traj, pd, sd, ctx->stream));
    ctx->launches++;
    if (!p_dev) TNQ_CUDA(cudaMemcpyAsync(p_out + base, stage, 8 * nv, cudaMemcpyDeviceToHost, ctx->stream));
    if (se_out && !se_dev)
      TNQ_CUDA(cudaMemcpyAsync(se_out + base, stage + per, 8 * nv, cudaMemcpyDeviceToHost, ctx->stream));
    if (!p_dev || (se_out && !se_dev)) TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return TNQ_OK;
  };
  // identical trajectories (most draws pick the identity-like operator A_0)
  // are contracted once and weighted by their number
  // (the draws of the last (seed, n_traj) are kept with the plan)
  if (p->dedup_seed != seed || p->dedup_n != n_traj || p->dedup_mult.empty()) {
    distinct_trajectories(p, seed, n_traj, &p->dedup_picks, &p->dedup_mult);
    p->dedup_seed = seed;
    p->dedup_n = n_traj;
  }
  p->last_distinct = (int64_t)p->dedup_mult.size();
  return noisy_driver(ctx, p, 0, n_traj, seed, n_bs, bits, consume, batch_end, &p->dedup_picks, &p->dedup_mult);
}

tnq_status exec_traj_amplitudes(Ctx* ctx, Plan* p, uint64_t seed, int64_t traj_begin, int64_t n_traj, int64_t n_bs,
                                const int8_t* bits, double* out) {
  tnq_status st = noisy_checks(p, n_traj, n_bs, bits, out);
  if (st != TNQ_OK || n_bs == 0) return st;
  if (traj_begin < 0) return fail(TNQ_ERR_INVALID_ARG, "traj_begin must be >= 0");
  TNQ_CUDA(cudaSetDevice(ctx->device));
  char* ws = static_cast<char*>(p->bound_ws);
  const bool out_dev = is_device_ptr(out);
  const int64_t per = int64_t(1) << p->batch_log2;
  double2* stage = reinterpret_cast<double2*>(ws + p->ws_out_stage);
  // Device output: one kernel writes the chunk.  Host output: the staging area
  // holds 2^batch_log2 complex values, so each trajectory row goes through it.
  auto consume = [&](int phase, int64_t base, int64_t nv, int64_t tb, int64_t nt, const std::vector<int>& bpos,
                     const std::vector<int>& tpos) -> tnq_status {
    if (phase < 0) return TNQ_OK;
    double2* o = reinterpret_cast<double2*>(out);
    if (out_dev) {
      TNQ_CUDA(launch_traj_amplitudes_out(ws + p->ws_acc, nv, 0, nt, bpos.data(), (int)bpos.size(), tpos.data(),
                                          (int)tpos.size(), o + tb * n_bs + base, n_bs, ctx->stream));
      ctx->launches++;
      return TNQ_OK;
    }
    for (int64_t j = 0; j < nt; ++j) {
      TNQ_CUDA(launch_traj_amplitudes_out(ws + p->ws_acc, nv, j, 1, bpos.data(), (int)bpos.size(), tpos.data(),
                                          (int)tpos.size(), stage, per, ctx->stream));
      ctx->launches++;
      TNQ_CUDA(cudaMemcpyAsync(o + (tb + j) * n_bs + base, stage, 16 * size_t(nv), cudaMemcpyDeviceToHost,
                               ctx->stream));
      TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return TNQ_OK;
  };
  auto batch_end = [&](int64_t, int64_t) -> tnq_status { return TNQ_OK; };
  return noisy_driver(ctx, p, traj_begin, n_traj, seed, n_bs, bits, consume, batch_end);
}

tnq_status exec_expectation(Ctx* ctx, Plan* p, const double* coeffs, double* value, double* term_values) {
  if (!p->bound_ws) return fail(TNQ_ERR_WORKSPACE, "plan has no bound workspace");
  if (!p->expectation) return fail(TNQ_ERR_INVALID_ARG, "plan is not an expectation-value plan");
  if (!coeffs || !value) return fail(TNQ_ERR_INVALID_ARG, "NULL coefficients or value");
  TNQ_CUDA(cudaSetDevice(ctx->device));
  char* ws = static_cast<char*>(p->bound_ws);
  int* err_flag = reinterpret_cast<int*>(ws + p->ws_misc);
  int8_t* bits_stage = reinterpret_cast<int8_t*>(ws + p->ws_bits);
  double2* stage = reinterpret_cast<double2*>(ws + p->ws_out_stage);
  const auto& rl = p->tensors[p->root].labels;
  std::vector<int> tpos;
  for (int l : p->net.traj_labels) tpos.push_back(int(std::find(rl.begin(), rl.end(), l) - rl.begin()));
  const int t = (int)tpos.size();
  const int64_t tper = int64_t(1) << t;
  const size_t acc_bytes = 16 * (size_t(1) << p->tensors[p->root].rank);
  const int n_slices = 1 << p->slice_labels.size();
  TNQ_CUDA(cudaMemsetAsync(err_flag, 0, 2 * sizeof(int), ctx->stream));
  // <0...0| closes every wire (the network is U, the Pauli operators, U^dagger)
  TNQ_CUDA(cudaMemsetAsync(bits_stage, 0, size_t(p->net.row_len), ctx->stream));
  TNQ_CUDA(fill_projections(ctx, proj_leaves(p, ws), 0, bits_stage, 1, err_flag));
  {
    tnq_status st = ensure_folded(ctx, p);
    if (st != TNQ_OK) return st;
  }
  std::vector<double> vals(size_t(p->n_terms));
  std::vector<double2> host(static_cast<size_t>(tper));
  // without selectors (every term the identity) one contraction serves all terms
  const int64_t step = p->n_sel > 0 ? tper : p->n_terms;
  for (int64_t tb = 0; tb < p->n_terms; tb += step) {
    const int64_t nt = std::min<int64_t>(tper, p->n_terms - tb);
    if (!p->traj_leaves.empty()) {
      TNQ_CUDA(launch_traj_leaves(reinterpret_cast<const TrajLeafDesc*>(ws + p->ws_traj), (int)p->traj_leaves.size(),
                                  reinterpret_cast<const TrajFactor*>(ws + p->ws_traj_factors),
                                  reinterpret_cast<const double2*>(ws + p->ws_traj_mats),
                                  reinterpret_cast<const double*>(ws + p->ws_traj_cumq), ws, 0, uint64_t(tb), t,
                                  ctx->stream, reinterpret_cast<const int8_t*>(ws + p->ws_picks), p->n_sel,
                                  p->n_terms));
      ctx->launches++;
    }
    TNQ_CUDA(launch_zero(ws + p->ws_acc, acc_bytes, ctx->stream));
    for (int s = 0; s < n_slices; ++s) {
      tnq_status st = run_pass(ctx, p, s, ws, s == 0);
      if (st != TNQ_OK) return st;
    }
    TNQ_CUDA(launch_traj_amplitudes_out(ws + p->ws_acc, 1, 0, nt, nullptr, 0, tpos.data(), t, stage, 1, ctx->stream));
    ctx->launches++;
    TNQ_CUDA(cudaMemcpyAsync(host.data(), stage, 16 * size_t(nt), cudaMemcpyDeviceToHost, ctx->stream));
    TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (p->n_sel > 0) {
      for (int64_t j = 0; j < nt; ++j) vals[size_t(tb + j)] = host[size_t(j)].x;
    } else {
      for (auto& v : vals) v = host[0].x;
    }
  }
  int herr[2] = {0, 0};
  TNQ_CUDA(cudaMemcpyAsync(herr, err_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->timing) {
    tnq_status ts = timing_collect(ctx);
    if (ts != TNQ_OK) return ts;
  }
  if (herr[1]) return fail(TNQ_ERR_TIMEOUT, "a tensor-core GEMM wait expired; results are invalid");
  double sum = 0.0;
  for (int64_t j = 0; j < p->n_terms; ++j) {
    sum += coeffs[j] * vals[size_t(j)];
    if (term_values) term_values[j] = vals[size_t(j)];
  }
  *value = sum;
  return TNQ_OK;
}

// Partial-product bytes any split of an output of 2^rc elements can need.
static size_t partial_bound(int rc) {
  double e = std::min(kPartialCapElems, std::ldexp(1.0, rc) * 1024.0);
  return size_t(8 * e);
}

size_t contract_workspace_bytes(int precision, int ra, int rb, int rc) {
  (void)precision;
  size_t na = size_t(1) << std::max(ra, rb), nb = na;
  return 32 * na + 16 * nb + 8 * (size_t(1) << rc) + partial_bound(rc) + 5 * 4096;
}

tnq_status exec_contract_pair(Ctx* ctx, const void* A, int ra, const int* al, const void* B, int rb,
                              const int* bl, void* C, int rc, const int* cl, void* ws, size_t ws_bytes) {
  if (ra < 0 || rb < 0 || rc < 0 || ra > 31 || rb > 31 || rc > 31)
    return fail(TNQ_ERR_INVALID_ARG, "ranks must be in [0, 31]");
  std::vector<int> la(al, al + ra), lb(bl, bl + rb), lc(cl, cl + rc);
  auto has = [](const std::vector<int>& v, int l) { return std::find(v.begin(), v.end(), l) != v.end(); };
  auto uniq = [](std::vector<int> v) {
    std::sort(v.begin(), v.end());
    return std::adjacent_find(v.begin(), v.end()) == v.end();
  };
  if (!uniq(la) || !uniq(lb) || !uniq(lc)) return fail(TNQ_ERR_INVALID_ARG, "repeated label within a tensor");
  for (int l : lc)
    if (!has(la, l) && !has(lb, l)) return fail(TNQ_ERR_INVALID_ARG, "output label missing from both operands");
  for (int l : la)
    if (!has(lb, l) && !has(lc, l)) return fail(TNQ_ERR_INVALID_ARG, "label of A neither shared nor kept");
  for (int l : lb)
    if (!has(la, l) && !has(lc, l)) return fail(TNQ_ERR_INVALID_ARG, "label of B neither shared nor kept");
  if (!ws || ws_bytes < contract_workspace_bytes(ctx->precision, ra, rb, rc))
    return fail(TNQ_ERR_WORKSPACE, "workspace too small for tnq_contract_pair");
  TNQ_CUDA(cudaSetDevice(ctx->device));
  // A side = operand with fewer elements; K and H orders follow the other one
  bool swap = ra > rb;
  const std::vector<int>& xa = swap ? lb : la;
  const std::vector<int>& xb = swap ? la : lb;
  const void* pa = swap ? B : A;
  const void* pb = swap ? A : B;
  std::vector<int> K, Hh, M, N;
  for (int l : xb)
    if (has(xa, l)) (has(lc, l) ? Hh : K).push_back(l);
  for (int l : xa)
    if (!has(xb, l)) M.push_back(l);
  for (int l : xb)
    if (!has(xa, l)) N.push_back(l);
  std::vector<int> a_req = K, b_req = K, out = N;
  a_req.insert(a_req.end(), M.begin(), M.end());
  a_req.insert(a_req.end(), Hh.begin(), Hh.end());
  b_req.insert(b_req.end(), N.begin(), N.end());
  b_req.insert(b_req.end(), Hh.begin(), Hh.end());
  out.insert(out.end(), M.begin(), M.end());
  out.insert(out.end(), Hh.begin(), Hh.end());
  char* w = static_cast<char*>(ws);
  size_t na = size_t(1) << std::max(ra, rb);
  char* sa = w;
  char* sb = w + ((32 * na + 4095) & ~size_t(4095));
  char* sc = sb + ((16 * na + 4095) & ~size_t(4095));
  int* err = reinterpret_cast<int*>(sc + ((8 * (size_t(1) << rc) + 4095) & ~size_t(4095)));
  char* part = reinterpret_cast<char*>(err) + 4096;
  TNQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  bool direct = out == lc;
  std::vector<int> none;
  tnq_status st = run_gemm_step(ctx, pa, xa, xa != a_req, pb, xb, xb != b_req, a_req, b_req, none, 0,
                                (int)Hh.size(), (int)M.size(), (int)N.size(), (int)K.size(), sa, sb,
                                direct ? C : (void*)sc, nullptr, err, part, size_t(sb - sa));
  if (st != TNQ_OK) return st;
  if (!direct) {
    PermDesc d;
    build_perm_desc(out.data(), (int)out.size(), lc.data(), rc, nullptr, 0, PM_C64, 0, &d);
    TNQ_CUDA(perm(ctx, d, sc, C, nullptr, 0, 16.0 * std::ldexp(1.0, rc)));
  }
  int herr = 0;
  TNQ_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  TNQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->timing) {
    tnq_status ts = timing_collect(ctx);
    if (ts != TNQ_OK) return ts;
  }
  if (herr) return fail(TNQ_ERR_TIMEOUT, "a tensor-core GEMM wait expired; results are invalid");
  return TNQ_OK;
}

}  // namespace tnq
