// The analyzer of randUTV by blocks (§3.2.4, the analysis stage): the list
// of tasks, each with the blocks it reads (In) and writes (Out), built from
// the update list of the algorithm written for algorithms-by-blocks (Fig. 2)
// with the QRs done by blocks (QR_AB, §3.2.2: a dense QR of the leading block
// of a block column, then a triangular-dense QR of the leading R with each
// block below it).  Also the I/O of the traditional dispatcher and of the
// dispatcher with an LRU cache of blocks (§3.2.4, the execution stage), on
// any prefix of the list.  Host code only.
//
// Order of the tasks of one block step k (tile indices; rows of tiles 0..Mt-1,
// columns 0..Nt-1), as the paper's 2 x 2 example lists them:
//   right transform (columns remain after block k):
//     G_i for i >= k; Y_j = sum_i A_ij^T G_i (i outer, j inner);
//     q times: Z_i = sum_j A_ij Y_j (j outer), Y_j = sum_i A_ij^T Z_i;
//     dense QR of Y_k, td QR of (Y_k, Y_j) for j > k;
//     A_rk Q for every tile row r (all m rows), then [A_rk A_rj] Q for j > k;
//     the same on the tile rows of V;
//   left transform (rows remain below block k):
//     dense QR of A_kk, td QR of (A_kk, A_ik) for i > k;
//     Q^T A_kj for j > k, then Q^T [A_kj; A_ij] for i > k, j > k;
//     U_rk Q, then [U_rk U_ri] Q (before the vectors in A_kk, A_ik are cleared);
//     Keep_upper_triang(A_kk), Set_to_zero(A_ik) for i > k;
//   small SVD of A_kk (P = U_s, Q = V_s) and its folds:
//     A_kj = P^T A_kj (j > k), A_ik = A_ik V_s (i < k), V_rk V_s, U_rk U_s.
#include <algorithm>
#include <cstring>

#include "ab.h"
#include "common.cuh"

namespace rutv {

const char* ab_op_name(int op) {
  static const char* names[OP_NOPS] = {
      "Generate_normal_random", "Gemm_tn_oz", "Gemm_tn_oo", "Gemm_nn_oz", "Gemm_nn_oo",
      "Comp_dense_QR", "Comp_td_QR", "Apply_right_Q_of_dense_QR", "Apply_right_Q_td_QR",
      "Apply_left_Qt_of_dense_QR", "Apply_left_Qt_of_td_QR", "Keep_upper_triang", "Set_to_zero",
      "Svd_of_block", "Gemm_abta", "Gemm_aabt", "Gemm_aab"};
  return (op >= 0 && op < OP_NOPS) ? names[op] : "?";
}

std::vector<int64_t> ab_tile_starts(int64_t extent, int64_t p, int64_t b) {
  std::vector<int64_t> s;
  for (int64_t x = 0; x < p; x += b) s.push_back(x);
  for (int64_t x = p; x < extent; x += b) s.push_back(x);
  s.push_back(extent);
  return s;
}

namespace {

struct Builder {
  std::vector<AbTask> t;
  int step = 0;
  void add(int op, std::initializer_list<int64_t> in, std::initializer_list<int64_t> out) {
    AbTask a;
    std::memset(&a, 0, sizeof a);
    a.op = op;
    a.step = step;
    a.nin = 0;
    for (int64_t x : in) a.in[a.nin++] = x;
    a.nout = 0;
    for (int64_t x : out) a.out[a.nout++] = x;
    t.push_back(a);
  }
};

int64_t A(int64_t i, int64_t j) { return ab_block(AB_A, i, j); }
int64_t U(int64_t i, int64_t j) { return ab_block(AB_U, i, j); }
int64_t V(int64_t i, int64_t j) { return ab_block(AB_V, i, j); }
int64_t G(int64_t i) { return ab_block(AB_G, i, 0); }
int64_t Y(int64_t j) { return ab_block(AB_Y, j, 0); }
int64_t Z(int64_t i) { return ab_block(AB_Z, i, 0); }
int64_t B(int64_t j) { return ab_block(AB_B, j, 0); }
int64_t C(int64_t i) { return ab_block(AB_C, i, 0); }
int64_t P(int64_t k) { return ab_block(AB_P, k, 0); }
int64_t Q(int64_t k) { return ab_block(AB_Q, k, 0); }

}  // namespace

std::vector<AbTask> ab_analyze(int64_t m, int64_t n, int64_t b, int q, bool want_u, bool want_v) {
  Builder bd;
  if (m < 1 || n < 1 || b < 1) return bd.t;
  const int64_t p = std::min(m, n);
  const int64_t Mt = (int64_t)ab_tile_starts(m, p, b).size() - 1;
  const int64_t Nt = (int64_t)ab_tile_starts(n, p, b).size() - 1;
  const int64_t steps = (p + b - 1) / b;
  for (int64_t k = 0; k < steps; ++k) {
    bd.step = (int)k;
    const bool right = k + 1 < Nt, left = k + 1 < Mt;
    if (right) {
      for (int64_t i = k; i < Mt; ++i) bd.add(OP_GEN, {}, {G(i)});
      for (int64_t i = k; i < Mt; ++i)
        for (int64_t j = k; j < Nt; ++j) {
          if (i == k) bd.add(OP_TN_OZ, {A(i, j), G(i)}, {Y(j)});
          else bd.add(OP_TN_OO, {A(i, j), G(i), Y(j)}, {Y(j)});
        }
      for (int it = 0; it < q; ++it) {
        for (int64_t j = k; j < Nt; ++j)
          for (int64_t i = k; i < Mt; ++i) {
            if (j == k) bd.add(OP_NN_OZ, {A(i, j), Y(j)}, {Z(i)});
            else bd.add(OP_NN_OO, {A(i, j), Y(j), Z(i)}, {Z(i)});
          }
        for (int64_t i = k; i < Mt; ++i)
          for (int64_t j = k; j < Nt; ++j) {
            if (i == k) bd.add(OP_TN_OZ, {A(i, j), Z(i)}, {Y(j)});
            else bd.add(OP_TN_OO, {A(i, j), Z(i), Y(j)}, {Y(j)});
          }
      }
      bd.add(OP_QR_DENSE, {Y(k)}, {Y(k), B(k)});
      for (int64_t j = k + 1; j < Nt; ++j) bd.add(OP_QR_TD, {Y(k), Y(j)}, {Y(k), Y(j), B(j)});
      for (int64_t r = 0; r < Mt; ++r) bd.add(OP_RIGHT_DENSE, {Y(k), B(k), A(r, k)}, {A(r, k)});
      for (int64_t j = k + 1; j < Nt; ++j)
        for (int64_t r = 0; r < Mt; ++r)
          bd.add(OP_RIGHT_TD, {Y(j), B(j), A(r, k), A(r, j)}, {A(r, k), A(r, j)});
      if (want_v) {
        for (int64_t r = 0; r < Nt; ++r) bd.add(OP_RIGHT_DENSE, {Y(k), B(k), V(r, k)}, {V(r, k)});
        for (int64_t j = k + 1; j < Nt; ++j)
          for (int64_t r = 0; r < Nt; ++r)
            bd.add(OP_RIGHT_TD, {Y(j), B(j), V(r, k), V(r, j)}, {V(r, k), V(r, j)});
      }
    }
    if (left) {
      bd.add(OP_QR_DENSE, {A(k, k)}, {A(k, k), C(k)});
      for (int64_t i = k + 1; i < Mt; ++i)
        bd.add(OP_QR_TD, {A(k, k), A(i, k)}, {A(k, k), A(i, k), C(i)});
      for (int64_t j = k + 1; j < Nt; ++j) bd.add(OP_LEFT_DENSE, {A(k, k), C(k), A(k, j)}, {A(k, j)});
      for (int64_t i = k + 1; i < Mt; ++i)
        for (int64_t j = k + 1; j < Nt; ++j)
          bd.add(OP_LEFT_TD, {A(i, k), C(i), A(k, j), A(i, j)}, {A(k, j), A(i, j)});
      if (want_u) {
        for (int64_t r = 0; r < Mt; ++r) bd.add(OP_RIGHT_DENSE, {A(k, k), C(k), U(r, k)}, {U(r, k)});
        for (int64_t i = k + 1; i < Mt; ++i)
          for (int64_t r = 0; r < Mt; ++r)
            bd.add(OP_RIGHT_TD, {A(i, k), C(i), U(r, k), U(r, i)}, {U(r, k), U(r, i)});
      }
      bd.add(OP_KEEP_UPPER, {A(k, k)}, {A(k, k)});
      for (int64_t i = k + 1; i < Mt; ++i) bd.add(OP_SET_ZERO, {}, {A(i, k)});
    }
    bd.add(OP_SVD, {A(k, k)}, {A(k, k), P(k), Q(k)});
    for (int64_t j = k + 1; j < Nt; ++j) bd.add(OP_ABTA, {P(k), A(k, j)}, {A(k, j)});
    for (int64_t i = 0; i < k; ++i) bd.add(OP_AABT, {A(i, k), Q(k)}, {A(i, k)});
    if (want_v)
      for (int64_t r = 0; r < Nt; ++r) bd.add(OP_AABT, {V(r, k), Q(k)}, {V(r, k)});
    if (want_u)
      for (int64_t r = 0; r < Mt; ++r) bd.add(OP_AAB, {U(r, k), P(k)}, {U(r, k)});
  }
  return bd.t;
}

AbIo ab_simulate(const std::vector<AbTask>& tasks, int64_t ntasks, int64_t cache_blocks,
                 std::vector<int64_t>* trace) {
  AbIo io;
  if (ntasks < 0 || ntasks > (int64_t)tasks.size()) ntasks = (int64_t)tasks.size();
  if (cache_blocks <= 0) {  // traditional: read every input, write every output
    for (int64_t t = 0; t < ntasks; ++t) {
      io.reads += tasks[t].nin;
      io.writes += tasks[t].nout;
    }
    return io;
  }
  std::vector<int64_t> slot(cache_blocks, -1), last(cache_blocks, -1);
  std::vector<char> dirty(cache_blocks, 0);
  auto find = [&](int64_t blk) -> int64_t {
    for (int64_t s = 0; s < cache_blocks; ++s)
      if (slot[s] == blk) return s;
    return -1;
  };
  for (int64_t t = 0; t < ntasks; ++t) {
    const AbTask& a = tasks[t];
    auto pinned = [&](int64_t blk) {
      for (int x = 0; x < a.nin; ++x)
        if (a.in[x] == blk) return true;
      for (int x = 0; x < a.nout; ++x)
        if (a.out[x] == blk) return true;
      return false;
    };
    // a free slot, else the least recently used block not used by this task
    // (lowest slot on ties), written back first when it was modified
    auto take = [&]() -> int64_t {
      for (int64_t s = 0; s < cache_blocks; ++s)
        if (slot[s] < 0) return s;
      int64_t best = -1;
      for (int64_t s = 0; s < cache_blocks; ++s)
        if (!pinned(slot[s]) && (best < 0 || last[s] < last[best])) best = s;
      if (best < 0) return -1;
      if (dirty[best]) ++io.writes;
      slot[best] = -1;
      dirty[best] = 0;
      return best;
    };
    for (int x = 0; x < a.nin; ++x) {
      int64_t s = find(a.in[x]);
      if (s < 0) {
        s = take();
        if (s < 0) { io.reads = io.writes = -1; return io; }
        slot[s] = a.in[x];
        ++io.reads;
      }
      last[s] = t;
    }
    for (int x = 0; x < a.nout; ++x) {
      int64_t s = find(a.out[x]);
      if (s < 0) {
        s = take();
        if (s < 0) { io.reads = io.writes = -1; return io; }
        slot[s] = a.out[x];
      }
      dirty[s] = 1;
      last[s] = t;
    }
    if (trace) trace->insert(trace->end(), slot.begin(), slot.end());
  }
  return io;
}

}  // namespace rutv

using namespace rutv;

extern "C" {

int64_t randutv_ab_tasks(int64_t m, int64_t n, int b, int q, int want_u, int want_v, int32_t* ops,
                         int32_t* steps, int64_t* operands, int64_t cap) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (b < 1) return -3;
  if (q < 0 || q > 16) return -4;
  const std::vector<AbTask> t = ab_analyze(m, n, b, q, want_u != 0, want_v != 0);
  const int64_t count = (int64_t)t.size();
  const int64_t k = std::min<int64_t>(cap > 0 ? cap : 0, count);
  for (int64_t i = 0; i < k; ++i) {
    if (ops) ops[i] = t[i].op;
    if (steps) steps[i] = t[i].step;
    if (operands) {
      int64_t* o = operands + 8 * i;
      for (int x = 0; x < 4; ++x) o[x] = x < t[i].nin ? t[i].in[x] : -1;
      for (int x = 0; x < 4; ++x) o[4 + x] = x < t[i].nout ? t[i].out[x] : -1;
    }
  }
  return count;
}

const char* randutv_ab_op_name(int op) { return ab_op_name(op); }

int randutv_ab_io(int64_t m, int64_t n, int b, int q, int want_u, int want_v, int64_t max_tasks,
                  int64_t cache_blocks, int64_t* reads, int64_t* writes, int64_t* trace) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (b < 1) return -3;
  if (q < 0 || q > 16) return -4;
  if (cache_blocks < 0) return -8;
  const std::vector<AbTask> t = ab_analyze(m, n, b, q, want_u != 0, want_v != 0);
  std::vector<int64_t> tr;
  const AbIo io = ab_simulate(t, max_tasks, cache_blocks, (trace && cache_blocks > 0) ? &tr : nullptr);
  if (io.reads < 0) return RANDUTV_EUNSUPPORTED;  // a task needs more blocks than the cache holds
  if (reads) *reads = io.reads;
  if (writes) *writes = io.writes;
  if (trace) std::copy(tr.begin(), tr.end(), trace);
  return 0;
}

}  // extern "C"
