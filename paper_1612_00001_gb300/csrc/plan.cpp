// Host planner of the Block Recursive Inversion sweep.
//
// The forward procedure of the paper (Sec. 3.1) performs no arithmetic: it
// splits a frame - an ordered list of block rows, an ordered list of block
// columns and a role A/B/C/D - into four frames by dropping the last or first
// block row and the last or first block column (Step 1, Eq. F_k-1), and puts
// the pivot block M_22 back at position (2,2) by exchanging the first two
// rows and/or columns of every frame of order >= 3 (Step 2 / Step i,
// Eq. F_k-1_ChangeM22).  The backward procedure (Sec. 3.2) reduces each
// 2x2-assembled frame by the Schur complement its role names: A -> (./D),
// B -> (./C), C -> (./B), D -> (./A) (Eqs. SchurofA-SchurofD, Phi_A-Phi_D).
//
// A frame's value depends only on its identity: the kept block row and
// column and the sets of eliminated block rows and columns.  The planner
// builds the recursion once, shares every frame that appears under several
// parents (the reuse across branches that Sec. 8 proposes), and orders the
// distinct frames by order (level), so that each level runs as a few grouped
// launches.
#include <algorithm>
#include <cstdint>
#include <map>
#include <stdexcept>
#include <tuple>
#include <unordered_map>

#include "mbinv_internal.h"

namespace mbinv {

namespace {

struct Key {
  int kr, kc;
  uint64_t rm, cm;
  bool operator==(const Key& o) const { return kr == o.kr && kc == o.kc && rm == o.rm && cm == o.cm; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = k.rm * 0x9E3779B97F4A7C15ull ^ (k.cm + 0x632BE59BD9B4E019ull + (k.rm << 7));
    h ^= (uint64_t)(k.kr * 1315423911u + k.kc) * 0xBF58476D1CE4E5B9ull;
    return (size_t)(h ^ (h >> 29));
  }
};

struct Builder {
  Plan* P;
  std::unordered_map<Key, int, KeyHash> memo;

  int visit(const std::vector<int>& rows, const std::vector<int>& cols, int role) {
    const int p = (int)rows.size();
    const int kr = (role == 0 || role == 1) ? rows.front() : rows.back();
    const int kc = (role == 0 || role == 2) ? cols.front() : cols.back();
    Key key{kr, kc, 0, 0};
    for (int t = 0; t < p; ++t) {
      if (rows[t] != kr) key.rm |= 1ull << rows[t];
      if (cols[t] != kc) key.cm |= 1ull << cols[t];
    }
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    const int id = (int)P->f.size();
    P->f.emplace_back();
    memo.emplace(key, id);
    PFrame fr;
    fr.order = p;
    fr.role = role;
    fr.krow = kr;
    fr.kcol = kc;
    if (p >= 3) {
      for (int ch = 0; ch < 4; ++ch) {
        // A: drop last row and last col; B: drop last row, first col;
        // C: drop first row, last col;  D: drop first row, first col.
        const int r0 = (ch >= 2) ? 1 : 0;
        const int c0 = (ch & 1) ? 1 : 0;
        std::vector<int> cr(rows.begin() + r0, rows.begin() + r0 + p - 1);
        std::vector<int> cc(cols.begin() + c0, cols.begin() + c0 + p - 1);
        if (p - 1 >= 3) {
          if (cr[0] == P->prow) std::swap(cr[0], cr[1]);
          if (cc[0] == P->pcol) std::swap(cc[0], cc[1]);
        }
        fr.child[ch] = visit(cr, cc, ch);
      }
      // (kept, left, pivot, right) by role: value = kept - left * pivot^-1 * right
      static const int KLPR[4][4] = {{0, 1, 3, 2},   // A: a - b d^-1 c
                                     {1, 0, 2, 3},   // B: b - a c^-1 d
                                     {2, 3, 1, 0},   // C: c - d b^-1 a
                                     {3, 2, 0, 1}};  // D: d - c a^-1 b
      fr.kept = fr.child[KLPR[role][0]];
      fr.left = fr.child[KLPR[role][1]];
      fr.piv = fr.child[KLPR[role][2]];
      fr.right = fr.child[KLPR[role][3]];
    }
    P->f[id] = fr;
    return id;
  }
};

}  // namespace

Plan build_plan(int k, int i, int j, bool pad_last) {
  if (k < 2 || k > 63 || i < 0 || j < 0 || i >= k || j >= k) throw std::invalid_argument("bad plan request");
  Plan P;
  P.k = k;
  P.i = i;
  P.j = j;
  // Root lists for block (i, j): (P M Q)^-1 = Q^T M^-1 P^T, so rows start
  // with j and columns with i; the other indices keep their order.  When the
  // last block is padding (k does not divide n) and the request does not
  // touch it, it is placed second in both lists: it is then the pivot index,
  // eliminated in every frame, so no frame keeps padded rows or columns.
  const int last = k - 1;
  if (pad_last && k >= 3 && i != last && j != last) {
    P.rows = {j, last};
    P.cols = {i, last};
    for (int x = 0; x < last; ++x)
      if (x != i && x != j) {
        P.rows.push_back(x);
        P.cols.push_back(x);
      }
    if (i != j) {
      P.rows.push_back(i);
      P.cols.push_back(j);
    }
  } else if (i == j) {
    P.rows.push_back(i);
    for (int x = 0; x < k; ++x)
      if (x != i) P.rows.push_back(x);
    P.cols = P.rows;
  } else {
    P.rows.push_back(j);
    P.cols.push_back(i);
    for (int x = 0; x < k; ++x)
      if (x != i && x != j) {
        P.rows.push_back(x);
        P.cols.push_back(x);
      }
    P.rows.push_back(i);
    P.cols.push_back(j);
  }
  P.prow = P.rows[1];
  P.pcol = P.cols[1];
  Builder B{&P, {}};
  B.visit(P.rows, P.cols, 0);
  P.level.assign(k + 1, {});
  for (int id = 0; id < (int)P.f.size(); ++id) P.level[P.f[id].order].push_back(id);
  P.leaves = P.level[2].size();
  P.nonleaf = P.f.size() - P.leaves;
  return P;
}

// ------------------------------------------------------------- schedule

namespace {

struct SlotPool {
  std::vector<int> free_list;
  int next = 0, live = 0, peak = 0;
  int get() {
    int s;
    if (!free_list.empty()) {
      s = free_list.back();
      free_list.pop_back();
    } else {
      s = next++;
    }
    peak = std::max(peak, ++live);
    return s;
  }
  void put(int s) {
    if (s < 0) return;
    free_list.push_back(s);
    --live;
  }
};

Ref mblk(int r, int c) {
  Ref x;
  x.kind = Ref::MBLK;
  x.r = r;
  x.c = c;
  return x;
}
Ref slot(int s) {
  Ref x;
  x.kind = Ref::SLOT;
  x.slot = s;
  return x;
}
Ref outref() {
  Ref x;
  x.kind = Ref::OUT;
  return x;
}

}  // namespace

Schedule build_schedule(const Plan& P, int zchunk) {
  Schedule S;
  SlotPool pool;
  std::vector<int> val(P.f.size(), -1);  // slot of each frame's value
  const int k = P.k;

  // ---- level 2 (Backward Step 1): every leaf pivots on P = M[prow, pcol]
  {
    const std::vector<int>& lv = P.level[2];
    Step inv;
    inv.kind = Step::INV;
    const int pinv = pool.get();
    InvOp io;
    io.src = mblk(P.prow, P.pcol);
    io.dst = slot(pinv);
    inv.inv.push_back(io);
    S.steps.push_back(inv);
    S.inv_units += 2;
    S.inversions += 1;
    S.max_inv_batch = std::max(S.max_inv_batch, 1);
    // T_c = P^-1 M[prow, c] for every distinct leaf column c
    std::map<int, int> tcol;
    for (int id : lv) tcol[P.f[id].kcol] = -1;
    Step g1;
    g1.kind = Step::GEMM;
    for (auto& kv : tcol) {
      kv.second = pool.get();
      GemmOp g;
      g.A = slot(pinv);
      g.B = mblk(P.prow, kv.first);
      g.C = slot(kv.second);
      g.alpha = 1.0;
      g.beta = 0.0;
      g1.gemm.push_back(g);
    }
    S.steps.push_back(g1);
    Step g2;
    g2.kind = Step::GEMM;
    for (int id : lv) {
      const PFrame& fr = P.f[id];
      val[id] = pool.get();
      GemmOp g;  // leaf = M[a,c] - M[a,pc] T_c
      g.A = mblk(fr.krow, P.pcol);
      g.B = slot(tcol[fr.kcol]);
      g.Cin = mblk(fr.krow, fr.kcol);
      g.C = slot(val[id]);
      g.alpha = -1.0;
      g.beta = 1.0;
      g2.gemm.push_back(g);
    }
    S.steps.push_back(g2);
    S.gemm_flops_units += 2.0 * (double)(tcol.size() + lv.size());
    pool.put(pinv);
    for (auto& kv : tcol) pool.put(kv.second);
  }

  // ---- levels 3..k (Backward Steps 2..k-1): X = kept - left * (piv^-1 * right)
  for (int p = 3; p <= k; ++p) {
    const std::vector<int>& lv = P.level[p];
    std::map<int, int> pinv;  // pivot frame -> slot of its inverse
    for (int id : lv) pinv[P.f[id].piv] = -1;
    Step inv;
    inv.kind = Step::INV;
    for (auto& kv : pinv) {
      kv.second = pool.get();
      InvOp io;
      io.src = slot(val[kv.first]);
      io.dst = slot(kv.second);
      io.frame = kv.first;
      inv.inv.push_back(io);
    }
    S.max_inv_batch = std::max(S.max_inv_batch, (int)inv.inv.size());
    S.inv_units += 2.0 * (double)pinv.size();
    S.inversions += pinv.size();
    S.steps.push_back(inv);
    for (int id : lv) val[id] = pool.get();
    const int nz = (zchunk > 0) ? std::min<int>(zchunk, (int)lv.size()) : (int)lv.size();
    std::vector<int> z(nz);
    for (int t = 0; t < nz; ++t) z[t] = pool.get();
    for (size_t c0 = 0; c0 < lv.size(); c0 += nz) {
      const size_t c1 = std::min(lv.size(), c0 + nz);
      Step g1, g2;
      g1.kind = g2.kind = Step::GEMM;
      for (size_t t = c0; t < c1; ++t) {
        const PFrame& fr = P.f[lv[t]];
        GemmOp a;  // Z = piv^-1 * right
        a.A = slot(pinv[fr.piv]);
        a.B = slot(val[fr.right]);
        a.C = slot(z[t - c0]);
        g1.gemm.push_back(a);
        GemmOp b;  // X = kept - left * Z
        b.A = slot(val[fr.left]);
        b.B = slot(z[t - c0]);
        b.Cin = slot(val[fr.kept]);
        b.C = slot(val[lv[t]]);
        b.alpha = -1.0;
        b.beta = 1.0;
        g2.gemm.push_back(b);
      }
      S.steps.push_back(g1);
      S.steps.push_back(g2);
    }
    S.gemm_flops_units += 4.0 * (double)lv.size();
    for (int t = 0; t < nz; ++t) pool.put(z[t]);
    for (auto& kv : pinv) pool.put(kv.second);
    for (int id : P.level[p - 1]) {
      pool.put(val[id]);
      val[id] = -1;
    }
  }

  // ---- root (Eq. blockmatrix_NxN): N = (root value)^-1
  {
    Step inv;
    inv.kind = Step::INV;
    InvOp io;
    io.src = slot(val[0]);
    io.dst = outref();
    io.frame = 0;
    inv.inv.push_back(io);
    S.steps.push_back(inv);
    S.inv_units += 2;
    S.inversions += 1;
  }
  S.nslots = pool.peak;
  S.frames = P.f.size();
  return S;
}

}  // namespace mbinv
