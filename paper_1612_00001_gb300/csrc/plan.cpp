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
// Within one request a frame's value depends only on its identity: the kept
// block row and column and the sets of eliminated block rows and columns, so
// the planner visits each identity once (the reuse across branches that
// Sec. 8 proposes).  Across requests - the k^2 runs of Sec. 5, or any group
// of blocks - frames are merged by what they compute: the same four operand
// frames (or, for a leaf, the same kept block and pivot block), so a merged
// frame rounds exactly as it would in each request alone.  The distinct
// frames are then ordered by order (level), so that each level runs as a few
// grouped launches, and the products piv^-1 * right that several frames
// share are formed once.
#include <algorithm>
#include <array>
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
  int prow = -1, pcol = -1;                    // pivot block of the current request
  std::unordered_map<Key, int, KeyHash> memo;  // identity -> frame, per request
  std::map<std::array<int, 5>, int> cons;      // computation -> frame, all requests

  int make(const std::array<int, 5>& ck, const PFrame& fr) {
    auto it = cons.find(ck);
    if (it != cons.end()) return it->second;
    const int id = (int)P->f.size();
    P->f.push_back(fr);
    cons.emplace(ck, id);
    return id;
  }

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
    PFrame fr;
    fr.order = p;
    int id;
    if (p >= 3) {
      int child[4];
      for (int ch = 0; ch < 4; ++ch) {
        // A: drop last row and last col; B: drop last row, first col;
        // C: drop first row, last col;  D: drop first row, first col.
        const int r0 = (ch >= 2) ? 1 : 0;
        const int c0 = (ch & 1) ? 1 : 0;
        std::vector<int> cr(rows.begin() + r0, rows.begin() + r0 + p - 1);
        std::vector<int> cc(cols.begin() + c0, cols.begin() + c0 + p - 1);
        if (p - 1 >= 3) {
          if (cr[0] == prow) std::swap(cr[0], cr[1]);
          if (cc[0] == pcol) std::swap(cc[0], cc[1]);
        }
        child[ch] = visit(cr, cc, ch);
      }
      // (kept, left, pivot, right) by role: value = kept - left * pivot^-1 * right
      static const int KLPR[4][4] = {{0, 1, 3, 2},   // A: a - b d^-1 c
                                     {1, 0, 2, 3},   // B: b - a c^-1 d
                                     {2, 3, 1, 0},   // C: c - d b^-1 a
                                     {3, 2, 0, 1}};  // D: d - c a^-1 b
      fr.kept = child[KLPR[role][0]];
      fr.left = child[KLPR[role][1]];
      fr.piv = child[KLPR[role][2]];
      fr.right = child[KLPR[role][3]];
      id = make({1, fr.kept, fr.left, fr.piv, fr.right}, fr);
    } else {
      fr.krow = kr;
      fr.kcol = kc;
      fr.prow = prow;
      fr.pcol = pcol;
      id = make({0, kr, kc, prow, pcol}, fr);
    }
    memo.emplace(key, id);
    return id;
  }
};

// Root lists for block (i, j): (P M Q)^-1 = Q^T M^-1 P^T, so rows start with
// j and columns with i; the other indices keep their order.  When the last
// block is padding (k does not divide n) and the request does not touch it,
// it is placed second in both lists: it is then the pivot index, eliminated
// in every frame, so no frame keeps padded rows or columns.
void root_lists(int k, int i, int j, bool pad_last, std::vector<int>* rows, std::vector<int>* cols) {
  const int last = k - 1;
  rows->clear();
  cols->clear();
  if (pad_last && k >= 3 && i != last && j != last) {
    *rows = {j, last};
    *cols = {i, last};
    for (int x = 0; x < last; ++x)
      if (x != i && x != j) {
        rows->push_back(x);
        cols->push_back(x);
      }
    if (i != j) {
      rows->push_back(i);
      cols->push_back(j);
    }
  } else if (i == j) {
    rows->push_back(i);
    for (int x = 0; x < k; ++x)
      if (x != i) rows->push_back(x);
    *cols = *rows;
  } else {
    rows->push_back(j);
    cols->push_back(i);
    for (int x = 0; x < k; ++x)
      if (x != i && x != j) {
        rows->push_back(x);
        cols->push_back(x);
      }
    rows->push_back(i);
    cols->push_back(j);
  }
}

}  // namespace

Plan build_plan(int k, const std::vector<std::pair<int, int>>& reqs, bool pad_last) {
  if (k < 2 || k > 63 || reqs.empty()) throw std::invalid_argument("bad plan request");
  Plan P;
  P.k = k;
  P.reqs = reqs;
  Builder B{&P};
  for (const auto& ij : reqs) {
    const int i = ij.first, j = ij.second;
    if (i < 0 || j < 0 || i >= k || j >= k) throw std::invalid_argument("bad plan request");
    std::vector<int> rows, cols;
    root_lists(k, i, j, pad_last, &rows, &cols);
    B.prow = rows[1];
    B.pcol = cols[1];
    B.memo.clear();
    P.roots.push_back(B.visit(rows, cols, 0));
    P.request_frames += B.memo.size();
  }
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
Ref outref(int r) {
  Ref x;
  x.kind = Ref::OUT;
  x.slot = r;
  return x;
}

}  // namespace

Schedule build_schedule(const Plan& P, int zchunk) {
  Schedule S;
  SlotPool pool;
  std::vector<int> val(P.f.size(), -1);  // slot of each frame's value
  const int k = P.k;
  S.nouts = (int)P.roots.size();

  // ---- level 2 (Backward Step 1): a leaf pivots on its request's block
  // P = M[prow, pcol]; every distinct pivot block is inverted once and every
  // distinct T = P^-1 M[prow, c] formed once
  {
    const std::vector<int>& lv = P.level[2];
    std::map<std::pair<int, int>, int> pinv;         // (prow, pcol) -> slot of P^-1
    std::map<std::tuple<int, int, int>, int> tcol;   // (prow, pcol, c) -> slot of T
    for (int id : lv) {
      const PFrame& fr = P.f[id];
      pinv[{fr.prow, fr.pcol}] = -1;
      tcol[std::make_tuple(fr.prow, fr.pcol, fr.kcol)] = -1;
    }
    Step inv;
    inv.kind = Step::INV;
    for (auto& kv : pinv) {
      kv.second = pool.get();
      InvOp io;
      io.src = mblk(kv.first.first, kv.first.second);
      io.dst = slot(kv.second);
      inv.inv.push_back(io);
    }
    S.steps.push_back(inv);
    S.inv_units += 2.0 * (double)pinv.size();
    S.inversions += pinv.size();
    S.max_inv_batch = std::max(S.max_inv_batch, (int)pinv.size());
    Step g1;
    g1.kind = Step::GEMM;
    for (auto& kv : tcol) {
      kv.second = pool.get();
      GemmOp g;
      g.A = slot(pinv[{std::get<0>(kv.first), std::get<1>(kv.first)}]);
      g.B = mblk(std::get<0>(kv.first), std::get<2>(kv.first));
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
      g.A = mblk(fr.krow, fr.pcol);
      g.B = slot(tcol[std::make_tuple(fr.prow, fr.pcol, fr.kcol)]);
      g.Cin = mblk(fr.krow, fr.kcol);
      g.C = slot(val[id]);
      g.alpha = -1.0;
      g.beta = 1.0;
      g2.gemm.push_back(g);
    }
    S.steps.push_back(g2);
    S.gemm_flops_units += 2.0 * (double)(tcol.size() + lv.size());
    for (auto& kv : pinv) pool.put(kv.second);
    for (auto& kv : tcol) pool.put(kv.second);
  }

  // ---- levels 3..k (Backward Steps 2..k-1): X = kept - left * Z with
  // Z = piv^-1 * right formed once per distinct (piv, right)
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
    // distinct Z keys in order of first use; the level's frames grouped by
    // their Z key so that a chunk of keys serves a contiguous run of frames
    std::map<std::pair<int, int>, int> zidx;
    std::vector<std::pair<int, int>> zkeys;
    for (int id : lv) {
      const std::pair<int, int> zk{P.f[id].piv, P.f[id].right};
      if (zidx.emplace(zk, (int)zkeys.size()).second) zkeys.push_back(zk);
    }
    std::vector<int> order(lv.begin(), lv.end());
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return zidx[{P.f[a].piv, P.f[a].right}] < zidx[{P.f[b].piv, P.f[b].right}];
    });
    const int nzk = (int)zkeys.size();
    const int nz = (zchunk > 0) ? std::min(zchunk, nzk) : nzk;
    std::vector<int> z(nz);
    for (int t = 0; t < nz; ++t) z[t] = pool.get();
    size_t f0 = 0;
    for (int c0 = 0; c0 < nzk; c0 += nz) {
      const int c1 = std::min(nzk, c0 + nz);
      Step g1, g2;
      g1.kind = g2.kind = Step::GEMM;
      for (int t = c0; t < c1; ++t) {
        GemmOp a;  // Z = piv^-1 * right
        a.A = slot(pinv[zkeys[t].first]);
        a.B = slot(val[zkeys[t].second]);
        a.C = slot(z[t - c0]);
        g1.gemm.push_back(a);
      }
      for (; f0 < order.size(); ++f0) {
        const PFrame& fr = P.f[order[f0]];
        const int t = zidx[{fr.piv, fr.right}];
        if (t >= c1) break;
        GemmOp b;  // X = kept - left * Z
        b.A = slot(val[fr.left]);
        b.B = slot(z[t - c0]);
        b.Cin = slot(val[fr.kept]);
        b.C = slot(val[order[f0]]);
        b.alpha = -1.0;
        b.beta = 1.0;
        g2.gemm.push_back(b);
      }
      S.steps.push_back(g1);
      S.steps.push_back(g2);
    }
    S.gemm_flops_units += 2.0 * (double)(nzk + lv.size());
    for (int t = 0; t < nz; ++t) pool.put(z[t]);
    for (auto& kv : pinv) pool.put(kv.second);
    for (int id : P.level[p - 1]) {
      pool.put(val[id]);
      val[id] = -1;
    }
  }

  // ---- roots (Eq. blockmatrix_NxN): N = (root value)^-1 for every request
  {
    Step inv;
    inv.kind = Step::INV;
    for (size_t r = 0; r < P.roots.size(); ++r) {
      InvOp io;
      io.src = slot(val[P.roots[r]]);
      io.dst = outref((int)r);
      io.frame = P.roots[r];
      inv.inv.push_back(io);
    }
    S.max_inv_batch = std::max(S.max_inv_batch, (int)inv.inv.size());
    S.steps.push_back(inv);
    S.inv_units += 2.0 * (double)P.roots.size();
    S.inversions += P.roots.size();
  }
  S.nslots = pool.peak;
  S.frames = P.f.size();
  S.request_frames = P.request_frames;
  return S;
}

}  // namespace mbinv

// ------------------------------------------------------- bounded schedule
//
// Values of a bounded run, each a b x b matrix: a block of M, the inverse of
// a leaf pivot block, T = P^-1 M[prow, c], a frame's value, the inverse of a
// frame used as a pivot, Z = piv^-1 right.  Each is computed once, in the
// order a depth-first walk from the roots asks for it; the slot allocation
// below then decides which of them wait on the host.

namespace mbinv {

namespace {

struct BVal {
  enum Kind : int { MB, PINV, T, F, FINV, Z } kind;
  int a = -1, b = -1, c = -1;  // MB (r, c); PINV (prow, pcol); T (prow, pcol, col); F/FINV frame; Z (piv, right)
};

struct BOp {
  int kind;         // 0 inverse, 1 product
  int out;          // value id, or -1 - r for the output of request r
  int in[3];        // inverse: in[0]; product: A, B, Cin (Cin may be -1)
  double alpha, beta;
};

struct Bounded {
  const Plan& P;
  std::vector<BVal> vals;
  std::map<std::array<int, 4>, int> ids;
  std::vector<char> done;
  std::vector<BOp> ops;

  explicit Bounded(const Plan& p) : P(p) {}

  int id(int kind, int a, int b = -1, int c = -1) {
    auto key = std::array<int, 4>{kind, a, b, c};
    auto it = ids.find(key);
    if (it != ids.end()) return it->second;
    BVal v;
    v.kind = (BVal::Kind)kind;
    v.a = a;
    v.b = b;
    v.c = c;
    vals.push_back(v);
    done.push_back(0);
    ids.emplace(key, (int)vals.size() - 1);
    return (int)vals.size() - 1;
  }

  void emit(int kind, int out, int i0, int i1, int i2, double alpha = 1.0, double beta = 0.0) {
    BOp o;
    o.kind = kind;
    o.out = out;
    o.in[0] = i0;
    o.in[1] = i1;
    o.in[2] = i2;
    o.alpha = alpha;
    o.beta = beta;
    ops.push_back(o);
  }

  // Makes value v available: its inputs first (depth first), then its op.
  void need(int v) {
    if (done[v]) return;
    done[v] = 1;
    const BVal x = vals[v];
    switch (x.kind) {
      case BVal::MB:
        return;  // read from M where it lives
      case BVal::PINV: {
        const int m = id(BVal::MB, x.a, x.b);
        need(m);
        emit(0, v, m, -1, -1);
        return;
      }
      case BVal::T: {
        const int pi = id(BVal::PINV, x.a, x.b), m = id(BVal::MB, x.a, x.c);
        need(pi);
        need(m);
        emit(1, v, pi, m, -1, 1.0, 0.0);
        return;
      }
      case BVal::FINV: {
        const int f = id(BVal::F, x.a);
        need(f);
        emit(0, v, f, -1, -1);
        return;
      }
      case BVal::Z: {
        // the right operand first, then the pivot and its inverse: the order
        // of the walk that keeps the fewest values alive at once
        const int pi = id(BVal::FINV, x.a), r = id(BVal::F, x.b);
        need(r);
        need(pi);
        emit(1, v, pi, r, -1, 1.0, 0.0);
        return;
      }
      case BVal::F: {
        const PFrame& fr = P.f[x.a];
        if (fr.order == 2) {  // leaf = M[a,c] - M[a,pc] T_c
          const int t = id(BVal::T, fr.prow, fr.pcol, fr.kcol);
          const int ma = id(BVal::MB, fr.krow, fr.pcol), mk = id(BVal::MB, fr.krow, fr.kcol);
          need(t);
          need(ma);
          need(mk);
          emit(1, v, ma, t, mk, -1.0, 1.0);
        } else {  // X = kept - left * Z
          const int z = id(BVal::Z, fr.piv, fr.right);
          const int kv = id(BVal::F, fr.kept), lv = id(BVal::F, fr.left);
          need(kv);
          need(lv);
          need(z);
          emit(1, v, lv, z, kv, -1.0, 1.0);
        }
        return;
      }
    }
  }
};

}  // namespace

bool build_bounded_schedule(const Plan& P, int slots, bool host_m, Schedule* out) {
  Bounded B(P);
  for (size_t r = 0; r < P.roots.size(); ++r) {
    const int f = B.id(BVal::F, P.roots[r]);
    B.need(f);
    B.emit(0, -1 - (int)r, f, -1, -1);
  }
  const int nv = (int)B.vals.size();
  // a value lives in a slot unless it is a block of a device-resident M
  auto slotted = [&](int v) { return v >= 0 && (B.vals[v].kind != BVal::MB || host_m); };
  // uses of every value, in op order
  std::vector<std::vector<int>> uses(nv);
  for (int t = 0; t < (int)B.ops.size(); ++t)
    for (int q = 0; q < 3; ++q)
      if (B.ops[t].in[q] >= 0) uses[B.ops[t].in[q]].push_back(t);
  std::vector<size_t> up(nv, 0);  // uses[v][up[v]] is v's next use
  auto next_use = [&](int v) { return up[v] < uses[v].size() ? uses[v][up[v]] : INT32_MAX; };

  Schedule S;
  S.bounded = true;
  S.nouts = (int)P.roots.size();
  std::vector<int> slot_of(nv, -1), host_of(nv, -1);
  std::vector<int> free_slots, free_host;
  for (int q = slots - 1; q >= 0; --q) free_slots.push_back(q);
  int host_next = 0, host_live = 0;
  std::vector<int> resident;  // values holding a slot
  auto ref_slot = [](int s) {
    Ref x;
    x.kind = Ref::SLOT;
    x.slot = s;
    return x;
  };
  auto push_copy = [&](const Ref& src, const Ref& dst) {
    if (S.steps.empty() || S.steps.back().kind != Step::COPY) {
      Step st;
      st.kind = Step::COPY;
      S.steps.push_back(st);
    }
    S.steps.back().copy.push_back(CopyOp{src, dst});
  };
  // a free slot, evicting the resident value needed again last if there is
  // none (held: values the current op uses, which stay)
  auto take_slot = [&](const int* held, int nheld) -> int {
    if (free_slots.empty()) {
      int victim = -1, far = -1;
      for (int v : resident) {
        bool h = false;
        for (int q = 0; q < nheld; ++q) h |= held[q] == v;
        if (h) continue;
        const int nu = next_use(v);
        if (nu > far) {
          far = nu;
          victim = v;
        }
      }
      if (victim < 0) return -1;
      if (next_use(victim) != INT32_MAX && B.vals[victim].kind != BVal::MB && host_of[victim] < 0) {
        int h;
        if (!free_host.empty()) {
          h = free_host.back();
          free_host.pop_back();
        } else {
          h = host_next++;
        }
        host_of[victim] = h;
        ++host_live;
        S.nspill = std::max(S.nspill, host_live);
        Ref d;
        d.kind = Ref::SPILL;
        d.slot = h;
        push_copy(ref_slot(slot_of[victim]), d);
        ++S.spills;
      }
      free_slots.push_back(slot_of[victim]);
      slot_of[victim] = -1;
      resident.erase(std::find(resident.begin(), resident.end(), victim));
    }
    const int s = free_slots.back();
    free_slots.pop_back();
    S.nslots = std::max(S.nslots, slots - (int)free_slots.size());
    return s;
  };
  auto release = [&](int v) {  // v has no use left
    if (slot_of[v] >= 0) {
      free_slots.push_back(slot_of[v]);
      slot_of[v] = -1;
      resident.erase(std::find(resident.begin(), resident.end(), v));
    }
    if (host_of[v] >= 0) {
      free_host.push_back(host_of[v]);
      host_of[v] = -1;
      --host_live;
    }
  };
  for (int t = 0; t < (int)B.ops.size(); ++t) {
    const BOp& o = B.ops[t];
    int held[4] = {o.in[0], o.in[1], o.in[2], o.out};
    // inputs into slots
    for (int q = 0; q < 3; ++q) {
      const int u = o.in[q];
      if (!slotted(u) || slot_of[u] >= 0) continue;
      const int s = take_slot(held, 4);
      if (s < 0) return false;
      Ref src;
      if (B.vals[u].kind == BVal::MB) {
        src.kind = Ref::HOSTM;
        src.r = B.vals[u].a;
        src.c = B.vals[u].b;
      } else {
        if (host_of[u] < 0) return false;  // a value is always computed before it is read
        src.kind = Ref::SPILL;
        src.slot = host_of[u];
      }
      push_copy(src, ref_slot(s));
      ++S.loads;
      slot_of[u] = s;
      resident.push_back(u);
    }
    int so = -1;
    if (o.out >= 0) {
      so = take_slot(held, 4);
      if (so < 0) return false;
    }
    auto ref_of = [&](int v) {
      Ref x;
      if (v < 0) return x;
      if (slotted(v)) return ref_slot(slot_of[v]);
      x.kind = Ref::MBLK;
      x.r = B.vals[v].a;
      x.c = B.vals[v].b;
      return x;
    };
    Ref dst;
    if (o.out >= 0) {
      dst = ref_slot(so);
    } else {
      dst.kind = Ref::OUT;
      dst.slot = -1 - o.out;
    }
    Step st;
    if (o.kind == 0) {
      st.kind = Step::INV;
      InvOp io;
      io.src = ref_of(o.in[0]);
      io.dst = dst;
      st.inv.push_back(io);
      S.inv_units += 2;
      S.inversions += 1;
    } else {
      st.kind = Step::GEMM;
      GemmOp g;
      g.A = ref_of(o.in[0]);
      g.B = ref_of(o.in[1]);
      g.Cin = ref_of(o.in[2]);
      g.C = dst;
      g.alpha = o.alpha;
      g.beta = o.beta;
      st.gemm.push_back(g);
      S.gemm_flops_units += 2;
    }
    S.steps.push_back(st);
    S.max_inv_batch = 1;
    // uses consumed; values with none left let go of their slot and host copy
    for (int q = 0; q < 3; ++q) {
      const int u = o.in[q];
      if (u < 0) continue;
      while (up[u] < uses[u].size() && uses[u][up[u]] <= t) ++up[u];
    }
    for (int q = 0; q < 3; ++q) {
      const int u = o.in[q];
      if (u >= 0 && next_use(u) == INT32_MAX) release(u);
    }
    if (o.out >= 0) {
      slot_of[o.out] = so;
      resident.push_back(o.out);
      if (next_use(o.out) == INT32_MAX) release(o.out);
    }
  }
  S.frames = P.f.size();
  S.request_frames = P.request_frames;
  *out = std::move(S);
  return true;
}

}  // namespace mbinv

// ----------------------------------------------- principal Schur variant
//
// The stability variant the paper names as future work (Sec. 8: a
// reformulation with respect to the Schur complement M/A of Eq. SchurofA):
// block (i, j) of M^-1 from principal pivots only.  With C the other block
// indices (ascending), each c in C is eliminated in turn from the current
// Schur complement S (initially M):
//     S[r][q] <- S[r][q] - S[r][c] (S[c][c]^-1 S[c][q])    for r, q not yet eliminated,
// leaving S over {i, j}, whose inverse holds N_ij:
//     i = j:  N_ii = S[i][i]^-1;
//     i != j: Z = S[i][i]^-1 S[i][j],  T = S[j][j] - S[j][i] Z,  N_ij = -Z T^-1.
// Every pivot is a principal Schur complement (nonsingular and well
// conditioned for diagonally dominant or SPD M), unlike the paper's
// non-principal frames; the work is (2/3) k^3 b^3 instead of the DAG's.

namespace mbinv {

Schedule build_psc_schedule(int k, int i, int j) {
  if (k < 2 || i < 0 || j < 0 || i >= k || j >= k) throw std::invalid_argument("bad variant request");
  Schedule S;
  SlotPool pool;
  std::vector<std::vector<Ref>> cur(k, std::vector<Ref>(k));
  for (int r = 0; r < k; ++r)
    for (int q = 0; q < k; ++q) cur[r][q] = mblk(r, q);
  std::vector<int> alive;  // blocks not yet eliminated, eliminated ones first in order
  std::vector<int> order;
  for (int x = 0; x < k; ++x)
    if (x != i && x != j) order.push_back(x);
  if (i == j) {
    alive = order;
    alive.push_back(i);
  } else {
    alive = order;
    alive.push_back(i);
    alive.push_back(j);
  }
  auto put = [&](const Ref& r) {
    if (r.kind == Ref::SLOT) pool.put(r.slot);
  };
  auto gemm = [&](Step& st, Ref A, Ref B, Ref Cin, Ref C, double alpha, double beta) {
    GemmOp g;
    g.A = A;
    g.B = B;
    g.Cin = Cin;
    g.C = C;
    g.alpha = alpha;
    g.beta = beta;
    st.gemm.push_back(g);
    S.gemm_flops_units += 2;
  };
  auto inv = [&](Ref src, Ref dst) {
    Step st;
    st.kind = Step::INV;
    InvOp io;
    io.src = src;
    io.dst = dst;
    st.inv.push_back(io);
    S.steps.push_back(st);
    S.inv_units += 2;
    S.inversions += 1;
  };
  const int nelim = (int)order.size();
  for (int t = 0; t < nelim; ++t) {
    const int c = order[t];
    std::vector<int> rest(alive.begin() + t + 1, alive.end());
    const Ref p = slot(pool.get());
    inv(cur[c][c], p);
    put(cur[c][c]);
    Step gz, gu;
    gz.kind = gu.kind = Step::GEMM;
    std::vector<Ref> z(k);
    for (int q : rest) {  // Z_q = S[c][c]^-1 S[c][q]
      z[q] = slot(pool.get());
      gemm(gz, p, cur[c][q], Ref(), z[q], 1.0, 0.0);
    }
    for (int r : rest)  // S[r][q] -= S[r][c] Z_q
      for (int q : rest) {
        const Ref out = cur[r][q].kind == Ref::SLOT ? cur[r][q] : slot(pool.get());
        gemm(gu, cur[r][c], z[q], cur[r][q], out, -1.0, 1.0);
        cur[r][q] = out;
      }
    S.steps.push_back(gz);
    S.steps.push_back(gu);
    put(p);
    for (int q : rest) {
      pool.put(z[q].slot);
      put(cur[c][q]);
      put(cur[q][c]);
    }
  }
  Ref outr;
  outr.kind = Ref::OUT;
  outr.slot = 0;
  if (i == j) {
    inv(cur[i][i], outr);
  } else {
    const Ref pi = slot(pool.get()), z = slot(pool.get()), tt = slot(pool.get()), ti = slot(pool.get());
    inv(cur[i][i], pi);
    Step g1, g2, g3;
    g1.kind = g2.kind = g3.kind = Step::GEMM;
    gemm(g1, pi, cur[i][j], Ref(), z, 1.0, 0.0);             // Z = S_ii^-1 S_ij
    S.steps.push_back(g1);
    gemm(g2, cur[j][i], z, cur[j][j], tt, -1.0, 1.0);        // T = S_jj - S_ji Z
    S.steps.push_back(g2);
    inv(tt, ti);                                             // T^-1
    gemm(g3, z, ti, Ref(), outr, -1.0, 0.0);                 // N_ij = -Z T^-1
    S.steps.push_back(g3);
  }
  S.nslots = pool.peak;
  S.max_inv_batch = 1;
  S.frames = S.request_frames = 0;
  return S;
}

}  // namespace mbinv
