// mechanism.cpp -- host-side mechanism compiler.
//
// Turns reaction tables (Background section of the paper: reactions
// c1 y1 + ... -> c_{m+1} y_{m+1} + ..., each adding -c_i r_j to its reactants
// and +c_i r_j to its products) into the device tables the solve kernels run:
//   * the net stoichiometry nu_ij and the f(y) gather (a2);
//   * the Jacobian pattern J_il = sum_j nu_ij dr_j/dy_l plus the diagonal (a3);
//   * a static Markowitz pivot order, the symbolic LU fill, and the warp
//     programs that form M = I - c J in the LU slots, factor it and run the
//     forward/back substitutions (a4, a5).
// The CVODE solver the paper names stores its Jacobian in a SPARSE matrix
// (Background section); here the sparse structure is analysed once per
// mechanism and baked into race-free 32-lane programs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <queue>

#include "internal.h"

namespace chemgpu {

namespace {

// ---------------------------------------------------------------- scheduler
// Places ops into passes of at most 32 so that no two ops of a pass touch the
// same location unless both only read it; ops keep the program order of every
// location they share, so any valid placement computes the same values.
//
// While a program is emitted, add() places each op first-fit into the earliest
// pass its operands allow (lastw / lastr: the pass that last wrote / read each
// location), which the emitters consult to shape their sums.  It also records
// every op with the earlier ops it must follow (the last writer of each
// operand and of its target, and the target's readers since that write).
// finish() then packs the recorded graph afresh by list scheduling: pass by
// pass it takes the ready ops with the longest remaining dependency chain
// first (a reciprocal weighs RECIP_WEIGHT, the FP64 instructions of its pass),
// and a pass holds reciprocals only when the most urgent ready op is one.
struct Scheduler {
  static constexpr int RECIP_WEIGHT = 4;
  std::vector<int> lastw, lastr;
  std::vector<std::vector<Op>> passes;
  std::vector<int> kind;
  int n_ops = 0;
  // the recorded program
  std::vector<Op> rec_op;
  std::vector<int> rec_kind;
  std::vector<std::vector<int>> rec_pred;
  std::vector<int> lw_op;                        // last writer op of each location
  std::vector<std::vector<int>> readers;         // its readers since that write
  explicit Scheduler(int n_loc) : lastw(n_loc, -1), lastr(n_loc, -1), lw_op(n_loc, -1), readers(n_loc) {}

  void add(const Op &op, int k, const int *reads, int nr, int write) {
    int e = 0;
    for (int i = 0; i < nr; ++i) e = std::max(e, lastw[reads[i]] + 1);
    e = std::max(e, lastw[write] + 1);
    e = std::max(e, lastr[write] + 1);
    int p = e;
    while (p < (int)passes.size() && (kind[p] != k || passes[p].size() >= (size_t)WARP)) ++p;
    if (p == (int)passes.size()) {
      passes.emplace_back();
      kind.push_back(k);
    }
    passes[p].push_back(op);
    for (int i = 0; i < nr; ++i) lastr[reads[i]] = std::max(lastr[reads[i]], p);
    lastw[write] = p;
    n_ops++;

    const int id = (int)rec_op.size();
    std::vector<int> pred;
    for (int i = 0; i < nr; ++i)
      if (lw_op[reads[i]] >= 0) pred.push_back(lw_op[reads[i]]);
    if (lw_op[write] >= 0) pred.push_back(lw_op[write]);
    for (int r : readers[write]) pred.push_back(r);
    std::sort(pred.begin(), pred.end());
    pred.erase(std::unique(pred.begin(), pred.end()), pred.end());
    for (int i = 0; i < nr; ++i)
      if (reads[i] != write) readers[reads[i]].push_back(id);
    readers[write].clear();
    lw_op[write] = id;
    rec_op.push_back(op);
    rec_kind.push_back(k);
    rec_pred.push_back(std::move(pred));
  }
  void fma(int t, int a, int b, int c) {
    const int r[3] = {a, b, c};
    add(Op{(uint16_t)t, (uint16_t)a, (uint16_t)b, (uint16_t)c}, 0, r, 3, t);
  }
  void recip(int t, int a) {
    const int r[1] = {a};
    add(Op{(uint16_t)(t | OP_RECIP), (uint16_t)a, 0, 0}, 1, r, 1, t);
  }
  // wide: ops may also be packed 64 at a time into pairs of passes (when at
  // least 64 are ready, all of them mutually independent)
  HostProgram finish(bool wide = false) const {
    const int n = (int)rec_op.size();
    std::vector<std::vector<int>> succ(n);
    std::vector<int> npred(n, 0);
    for (int i = 0; i < n; ++i)
      for (int q : rec_pred[i]) {
        succ[q].push_back(i);
        npred[i]++;
      }
    // remaining weighted chain length; successors come later in program order
    std::vector<long> height(n, 0);
    for (int i = n - 1; i >= 0; --i) {
      long h = 0;
      for (int s2 : succ[i]) h = std::max(h, height[s2]);
      height[i] = h + (rec_kind[i] ? RECIP_WEIGHT : 1);
    }
    // ready ops per kind, most urgent first (then program order)
    auto later = [&](int a, int b) { return height[a] != height[b] ? height[a] < height[b] : a > b; };
    std::priority_queue<int, std::vector<int>, decltype(later)> ready[2] = {
        std::priority_queue<int, std::vector<int>, decltype(later)>(later),
        std::priority_queue<int, std::vector<int>, decltype(later)>(later)};
    for (int i = 0; i < n; ++i)
      if (npred[i] == 0) ready[rec_kind[i]].push(i);
    HostProgram hp;
    std::vector<int> pass;
    int done = 0;
    while (done < n) {
      int k;
      if (ready[0].empty()) k = 1;
      else if (ready[1].empty()) k = 0;
      else k = later(ready[0].top(), ready[1].top()) ? 1 : 0;
      pass.clear();
      const size_t width = (wide && k == 0 && ready[0].size() >= 2 * (size_t)WARP) ? 2 * WARP : WARP;
      while (!ready[k].empty() && pass.size() < width) {
        pass.push_back(ready[k].top());
        ready[k].pop();
      }
      // wide: a pass of reciprocals takes the most urgent ready FMAs into its
      // other lanes (the kernels run such a pass as one mixed op per lane)
      while (wide && k == 1 && !ready[0].empty() && pass.size() < (size_t)WARP) {
        pass.push_back(ready[0].top());
        ready[0].pop();
      }
      for (int i : pass) hp.ops.push_back(rec_op[i]);
      for (size_t i = pass.size(); i < (size_t)WARP; ++i) hp.ops.push_back(Op{OP_EMPTY, 0, 0, 0});
      if (k == 1) hp.unit.push_back(3);
      else if (width == WARP) hp.unit.push_back(0);
      else hp.unit.insert(hp.unit.end(), {1, 2});
      done += (int)pass.size();
      for (int i : pass)
        for (int s2 : succ[i])
          if (--npred[s2] == 0) ready[rec_kind[s2]].push(s2);
    }
    hp.n_ops = n_ops;
    return hp;
  }
};

// ------------------------------------------------------------- bank layout
// Shared memory serves a warp's access in wavefronts: one distinct 4-byte word
// per bank (32 banks) per wavefront.  Measured on GB300 with a pass
// interpreter at 4-16 warps per SM: an 8-byte access is served per half-warp
// (lanes 0-15, then 16-31), each half taking as many wavefronts as its most
// loaded bank pair (distinct doubles with equal slot index mod 16); random
// slots cost 6.4 wavefronts per operand and a pass 23 SM cycles, slots spread
// over the bank pairs two per operand 17 cycles (the pass's FP64 FMA alone
// needs 16).  The compiler numbers the LU slots row by row and fills a pass
// with whatever ops are ready, so the slots of a pass's operands collide in
// banks.  Two searches spread them, keeping every op in its pass (the
// programs compute the same values):
//  * lanes: per pass, swaps of ops between the half-warps that lower the
//    8-byte cost (per operand and half, the most loaded bank pair);
//  * slots: a permutation of the LU region by simulated annealing over swaps
//    of two slots' positions, lowering the number of pairs of distinct slots
//    that share a bank pair within a half (8-byte form) or a bank within the
//    whole pass (4-byte form, half weight), summed over the four operands of
//    every pass of the programs on WL weighted by how often each runs.
// The lanes are searched once for the slots as numbered and again for the
// permuted ones.  Both searches are deterministic (a fixed-seed generator).
struct BankProg {
  HostProgram *hp;
  double w;            // runs per factorisation of M
};

uint32_t xorshift(uint32_t &s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

// element of role r (0 t, 1 a, 2 b, 3 c) of an op as the device runs it (-1: no access)
int role_elem(const Op &o, bool recip, int r, int dummy, int zero, int one) {
  if (o.t == OP_EMPTY) {
    if (recip) return r == 0 ? dummy : r == 1 ? one : -1;
    return r == 0 ? dummy : zero;
  }
  if (o.t & OP_RECIP) return r == 0 ? (o.t & 0x7fff) : r == 1 ? o.a : -1;
  return r == 0 ? o.t : r == 1 ? o.a : r == 2 ? o.b : o.c;
}

bool recip_pass(const HostProgram &hp, int p) {
  for (int l = 0; l < WARP; ++l) {
    const Op &o = hp.ops[(size_t)p * WARP + l];
    if (o.t != OP_EMPTY && (o.t & OP_RECIP)) return true;
  }
  return false;
}

// The slot search: a permutation of the slots [0, n_perm) (perm[e] = new
// position of e), improved in place.  A group is the distinct slots of one
// operand of one pass, per half-warp in the pass's current lane order (16 bank
// pairs: position mod 16) and whole (32 banks: position mod 32).
void bank_permutation(const std::vector<BankProg> &progs, int n_perm, int dummy, int zero, int one, long iters,
                      std::vector<int> &perm) {
  constexpr int NB = 32;
  if (n_perm < 2 * NB) return;
  auto posof = [&](int e) { return e < n_perm ? perm[e] : e; };
  std::vector<float> gw;
  std::vector<uint8_t> cnt, gnb;     // [G][NB] counts, bins of each group
  std::vector<std::vector<int>> egroups(n_perm);   // groups of each permuted slot
  auto add_group = [&](std::vector<int> &els, float w, int nb) {
    std::sort(els.begin(), els.end());
    els.erase(std::unique(els.begin(), els.end()), els.end());
    bool any = false;
    for (int e : els) any |= e < n_perm;
    if (!any || els.size() < 2) return;
    const int g = (int)gw.size();
    gw.push_back(w);
    gnb.push_back((uint8_t)nb);
    cnt.resize(cnt.size() + NB, 0);
    for (int e : els) {
      cnt[(size_t)g * NB + posof(e) % nb]++;
      if (e < n_perm) egroups[e].push_back(g);
    }
  };
  for (const BankProg &bp : progs) {
    const HostProgram &hp = *bp.hp;
    for (int p = 0; p < hp.n_pass(); ++p) {
      const bool rc = recip_pass(hp, p);
      for (int r = 0; r < 4; ++r) {
        std::vector<int> whole;
        for (int h = 0; h < 2; ++h) {
          std::vector<int> half;
          for (int l = 16 * h; l < 16 * h + 16; ++l) {
            const int e = role_elem(hp.ops[(size_t)p * WARP + l], rc, r, dummy, zero, one);
            if (e >= 0) half.push_back(e);
          }
          whole.insert(whole.end(), half.begin(), half.end());
          add_group(half, (float)bp.w, 16);
        }
        add_group(whole, (float)(0.5 * bp.w), 32);
      }
    }
  }
  const int G = (int)gw.size();
  if (G == 0) return;
  std::vector<int> stamp(G, -1);
  uint32_t rng = 0x9e3779b9u;
  auto move = [&](int g, int pfrom, int pto) {
    cnt[(size_t)g * NB + pfrom % gnb[g]]--;
    cnt[(size_t)g * NB + pto % gnb[g]]++;
  };
  // Objective: pairs of distinct slots sharing a bank within a group (weighted);
  // it falls with every collision resolved, which the most loaded bank alone
  // does not show.  Simulated annealing over swaps of two slots' positions.
  auto pairs_delta = [&](int g, int pfrom, int pto) {
    const uint8_t *c = &cnt[(size_t)g * NB];
    const int bf = pfrom % gnb[g], bt = pto % gnb[g];
    if (bf == bt) return 0;
    return (int)c[bt] - ((int)c[bf] - 1);
  };
  double temp = 2.0;
  const double cool = std::pow(0.01 / temp, 1.0 / (double)std::max<long>(iters, 1));
  for (long it = 0; it < iters; ++it, temp *= cool) {
    const int e1 = (int)(xorshift(rng) % (uint32_t)n_perm);
    const int e2 = (int)(xorshift(rng) % (uint32_t)n_perm);
    if (e1 == e2) continue;
    const int p1 = perm[e1], p2 = perm[e2];
    const int tag = (int)(it & 0x3fffffff);
    for (int g : egroups[e1]) stamp[g] = tag;
    for (int g : egroups[e2])
      if (stamp[g] == tag) stamp[g] = -2;               // holds both: its counts do not change
    double delta = 0.0;
    for (int g : egroups[e1])
      if (stamp[g] == tag) delta += gw[g] * pairs_delta(g, p1, p2);
    for (int g : egroups[e2])
      if (stamp[g] != -2) delta += gw[g] * pairs_delta(g, p2, p1);
    // (a group of e1 and a group of e2 never coincide here, so the deltas add)
    bool accept = delta <= 0.0;
    if (!accept) accept = (double)(xorshift(rng) & 0xffffff) < 16777216.0 * std::exp(-delta / temp);
    if (accept) {
      for (int g : egroups[e1])
        if (stamp[g] == tag) move(g, p1, p2);
      for (int g : egroups[e2])
        if (stamp[g] != -2) move(g, p2, p1);
      perm[e1] = p2;
      perm[e2] = p1;
    }
    for (int g : egroups[e2]) stamp[g] = -1;
    for (int g : egroups[e1]) stamp[g] = -1;
  }
}

// 8-byte wavefronts of one pass with its ops in the given lane order
int half_cost(const std::vector<int> (&el)[4], const std::vector<int> &lane_op) {
  int cost = 0;
  for (int r = 0; r < 4; ++r)
    for (int h = 0; h < 2; ++h) {
      int e[16], n = 0;
      for (int l = 16 * h; l < 16 * h + 16; ++l) {
        const int x = el[r][lane_op[l]];
        if (x >= 0) e[n++] = x;
      }
      std::sort(e, e + n);
      n = (int)(std::unique(e, e + n) - e);
      int c[16] = {0}, m = 0;
      for (int i = 0; i < n; ++i) m = std::max(m, ++c[e[i] % 16]);
      cost += m;
    }
  return cost;
}

// The lane search over every pass of hp.
void bank_lanes(HostProgram &hp, int dummy, int zero, int one) {
  for (int p = 0; p < hp.n_pass(); ++p) {
    const bool rc = recip_pass(hp, p);
    Op *ops = &hp.ops[(size_t)p * WARP];
    std::vector<int> el[4];
    for (int r = 0; r < 4; ++r)
      for (int l = 0; l < WARP; ++l) el[r].push_back(role_elem(ops[l], rc, r, dummy, zero, one));
    std::vector<int> lane_op(WARP);
    for (int l = 0; l < WARP; ++l) lane_op[l] = l;
    int best = half_cost(el, lane_op);
    for (int round = 0; round < 8; ++round) {
      bool improved = false;
      for (int i = 0; i < 16; ++i)
        for (int j = 16; j < WARP; ++j) {
          std::swap(lane_op[i], lane_op[j]);
          const int c = half_cost(el, lane_op);
          if (c < best) {
            best = c;
            improved = true;
          } else {
            std::swap(lane_op[i], lane_op[j]);
          }
        }
      if (!improved) break;
    }
    Op tmp[WARP];
    for (int l = 0; l < WARP; ++l) tmp[l] = ops[lane_op[l]];
    for (int l = 0; l < WARP; ++l) ops[l] = tmp[l];
  }
}

// target = (fresh ? 0 : target) + sum_k W[coef_k] * W[src_k], split into chunks
// of at most L terms accumulated in separate temporaries and then combined.
void add_sum(Scheduler &s, int target, bool fresh, const std::vector<std::pair<int, int>> &terms,
             int L, int &temp_next, int ZERO, int ONE) {
  if (terms.empty()) {
    if (fresh) s.fma(target, ZERO, ZERO, ZERO);
    return;
  }
  std::vector<int> temps;
  for (size_t c0 = 0; c0 < terms.size(); c0 += L) {
    const size_t c1 = std::min(terms.size(), c0 + (size_t)L);
    int acc;
    bool first_fresh;
    if (c0 == 0) {
      acc = target;
      first_fresh = fresh;
    } else {
      acc = temp_next++;
      temps.push_back(acc);
      first_fresh = true;
    }
    for (size_t k = c0; k < c1; ++k) {
      const int c = (k == c0 && first_fresh) ? ZERO : acc;
      s.fma(acc, terms[k].first, terms[k].second, c);
    }
  }
  for (int t : temps) s.fma(target, ONE, t, target);
}

// Rows of a triangular solve: W[x_i] += sum W[coef] * W[x_k] over the row's
// terms (coef, k), rows emitted in the given order so every source is final
// first.  A row's terms are taken in the order their sources become final (the
// scheduler's last write), in the row itself or, when that finishes the row
// sooner, split with one temporary from a small pool that is folded in last.
void emit_rows(Scheduler &s, const std::vector<int> &rows, const std::vector<std::vector<std::pair<int, int>>> &terms,
               const std::vector<int> &xloc, int tmp0, int ntmp, int &tnext, int ZERO, int ONE) {
  for (int i : rows) {
    std::vector<std::pair<int, int>> tk = terms[i];
    if (tk.empty()) continue;
    const int x = xloc[i];
    std::stable_sort(tk.begin(), tk.end(), [&](const std::pair<int, int> &a, const std::pair<int, int> &b) {
      return s.lastw[xloc[a.second]] < s.lastw[xloc[b.second]];
    });
    // earliest completion with the row alone, and with the row plus a temporary
    int t1 = s.lastw[x] + 1;
    for (auto &t : tk) t1 = std::max(t1, s.lastw[xloc[t.second]] + 1) + 1;
    int fx = s.lastw[x] + 1, ft = 0;
    std::vector<int> where(tk.size());
    bool used_t = false;
    for (size_t q = 0; q < tk.size(); ++q) {
      const int r = s.lastw[xloc[tk[q].second]] + 1;
      const int ex = std::max(fx, r), et = std::max(ft, r);
      if (et < ex) {
        where[q] = 1;
        ft = et + 1;
        used_t = true;
      } else {
        where[q] = 0;
        fx = ex + 1;
      }
    }
    const int t2 = used_t ? std::max(fx, ft) + 1 : fx;
    if (!used_t || t2 >= t1) {
      for (auto &t : tk) s.fma(x, t.first, xloc[t.second], x);
      continue;
    }
    const int tmp = tmp0 + (tnext++ % ntmp);
    bool fresh = true;
    for (size_t q = 0; q < tk.size(); ++q) {
      if (where[q]) {
        s.fma(tmp, tk[q].first, xloc[tk[q].second], fresh ? ZERO : tmp);
        fresh = false;
      } else {
        s.fma(x, tk[q].first, xloc[tk[q].second], x);
      }
    }
    s.fma(x, ONE, tmp, x);
  }
}

std::vector<int> markowitz_order(int S, std::vector<uint8_t> B) {
  std::vector<int> order;
  std::vector<uint8_t> alive(S, 1);
  for (int step = 0; step < S; ++step) {
    long best = -1;
    int bv = -1;
    for (int v = 0; v < S; ++v) {
      if (!alive[v]) continue;
      long r = 0, c = 0;
      for (int u = 0; u < S; ++u) {
        if (!alive[u] || u == v) continue;
        r += B[v * S + u];
        c += B[u * S + v];
      }
      const long score = r * c;
      if (bv < 0 || score < best) { best = score; bv = v; }
    }
    order.push_back(bv);
    for (int a = 0; a < S; ++a) {
      if (!alive[a] || a == bv || !B[a * S + bv]) continue;
      for (int b = 0; b < S; ++b)
        if (alive[b] && b != bv && B[bv * S + b]) B[a * S + b] = 1;
    }
    alive[bv] = 0;
  }
  return order;
}

struct ConstTable {
  std::map<double, int> idx;
  std::vector<double> vals;
  int base = 0;
  int get(double v) {
    auto it = idx.find(v);
    if (it != idx.end()) return it->second;
    const int i = base + (int)vals.size();
    idx[v] = i;
    vals.push_back(v);
    return i;
  }
};

constexpr int CHUNK = 8;
constexpr int X_VIRTUAL = 0x5000;   // the solve programs' name for the solve vector's slot 0 (above every WL slot)
constexpr int P_VIRTUAL = 0x6000;   // the M program's name for pair product 0 (above every WL slot)
constexpr int NSTMP = 16;   // temporaries of the triangular solves

}  // namespace

int compile_mechanism(int S, int R, const chem_reaction *rx, Mechanism &m, std::string &msg) {
  if (S < 1 || S > CHEM_MAX_SPECIES) { msg = "n_species must be in 1..128"; return CHEM_EINVAL; }
  if (R < 0 || R > 16384) { msg = "n_reactions must be in 0..16384"; return CHEM_EINVAL; }
  if (R > 0 && !rx) { msg = "reaction table is NULL"; return CHEM_EINVAL; }
  for (int j = 0; j < R; ++j) {
    const chem_reaction &r = rx[j];
    if (r.kind < CHEM_THERMAL || r.kind > CHEM_FALLOFF_SUM) { msg = "reaction " + std::to_string(j) + ": bad kind"; return CHEM_EINVAL; }
    if (r.n_reac < 1 || r.n_reac > CHEM_MAX_REAC) { msg = "reaction " + std::to_string(j) + ": n_reac must be 1..3"; return CHEM_EINVAL; }
    if (r.n_prod < 0 || r.n_prod > CHEM_MAX_PROD) { msg = "reaction " + std::to_string(j) + ": n_prod must be 0..8"; return CHEM_EINVAL; }
    for (int s = 0; s < r.n_reac; ++s)
      if (r.reac[s] < 0 || r.reac[s] >= S) { msg = "reaction " + std::to_string(j) + ": reactant index out of range"; return CHEM_EINVAL; }
    for (int p = 0; p < r.n_prod; ++p) {
      if (r.prod[p] < 0 || r.prod[p] >= S) { msg = "reaction " + std::to_string(j) + ": product index out of range"; return CHEM_EINVAL; }
      if (!std::isfinite(r.yield[p])) { msg = "reaction " + std::to_string(j) + ": non-finite yield"; return CHEM_EINVAL; }
    }
    if (r.kind != CHEM_PHOTOLYSIS && !(std::isfinite(r.A) && std::isfinite(r.Ea_over_R) && std::isfinite(r.B))) {
      msg = "reaction " + std::to_string(j) + ": non-finite Arrhenius parameters"; return CHEM_EINVAL;
    }
    if ((r.kind == CHEM_TROE || r.kind == CHEM_PRESSURE_SUM || r.kind == CHEM_FALLOFF_SUM) &&
        !(std::isfinite(r.A2) && std::isfinite(r.Ea2_over_R) && std::isfinite(r.B2))) {
      msg = "reaction " + std::to_string(j) + ": non-finite second Arrhenius term"; return CHEM_EINVAL;
    }
    if (r.kind == CHEM_FALLOFF_SUM && !(std::isfinite(r.A3) && std::isfinite(r.Ea3_over_R) && std::isfinite(r.B3))) {
      msg = "reaction " + std::to_string(j) + ": non-finite third Arrhenius term"; return CHEM_EINVAL;
    }
    if ((r.kind == CHEM_TROE || r.kind == CHEM_FALLOFF_SUM) && !(r.A2 > 0.0)) {
      msg = "reaction " + std::to_string(j) + ": the high-pressure limit needs A2 > 0"; return CHEM_EINVAL;
    }
    if (r.kind == CHEM_TROE && !(r.Fc > 0.0 && r.Fc <= 1.0 && r.N > 0.0 && std::isfinite(r.N))) {
      msg = "reaction " + std::to_string(j) + ": Troe needs Fc in (0, 1] and N > 0"; return CHEM_EINVAL;
    }
    if (r.kind == CHEM_PHOTOLYSIS && !std::isfinite(r.J)) { msg = "reaction " + std::to_string(j) + ": non-finite J"; return CHEM_EINVAL; }
  }
  m.S = S;
  m.R = R;
  m.rx.assign(rx, rx + R);
  m.max_reac = 1;
  m.n_phot = 0;
  for (int j = 0; j < R; ++j) {
    m.max_reac = std::max(m.max_reac, (int)rx[j].n_reac);
    m.n_phot += rx[j].kind == CHEM_PHOTOLYSIS;
  }

  // net stoichiometry nu_ij (reaction j, species i), in species order per reaction
  std::vector<std::vector<std::pair<int, double>>> nu(R);
  for (int j = 0; j < R; ++j) {
    std::map<int, double> acc;
    for (int s = 0; s < rx[j].n_reac; ++s) acc[rx[j].reac[s]] -= 1.0;
    for (int p = 0; p < rx[j].n_prod; ++p) acc[rx[j].prod[p]] += rx[j].yield[p];
    for (auto &kv : acc)
      if (kv.second != 0.0) nu[j].push_back(kv);
  }

  // Jacobian pattern (original species order) with the diagonal
  std::vector<uint8_t> P(S * S, 0);
  for (int i = 0; i < S; ++i) P[i * S + i] = 1;
  int n_pairs = 0;
  for (int j = 0; j < R; ++j)
    for (int s = 0; s < rx[j].n_reac; ++s) {
      n_pairs++;
      const int l = rx[j].reac[s];
      for (auto &kv : nu[j]) P[kv.first * S + l] = 1;
    }
  m.n_pairs = n_pairs;
  m.nnz_jac = 0;
  for (uint8_t v : P) m.nnz_jac += v;

  // static pivot order and symbolic fill in pivot order
  const std::vector<int> order = markowitz_order(S, P);
  m.pos.assign(S, 0);
  for (int k = 0; k < S; ++k) m.pos[order[k]] = k;
  std::vector<uint8_t> F(S * S, 0);
  for (int i = 0; i < S; ++i)
    for (int l = 0; l < S; ++l)
      if (P[i * S + l]) F[m.pos[i] * S + m.pos[l]] = 1;
  for (int k = 0; k < S; ++k)
    for (int i = k + 1; i < S; ++i) {
      if (!F[i * S + k]) continue;
      for (int j = k + 1; j < S; ++j)
        if (F[k * S + j]) F[i * S + j] = 1;
    }
  m.fill = F;
  std::vector<int> slot(S * S, -1);
  int nnz = 0;
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j)
      if (F[i * S + j]) slot[i * S + j] = nnz++;
  m.nnz_lu = nnz;

  // ---- per-cell array layouts
  // Wd (double): y[S], ONE, ZERO, nu constants of the f program, kt[R], rates[R],
  // f[S], f temps; the Jacobian's pair products (in the LU precision) reuse the
  // slots from rates[0] on while M is formed (rates, f and the f temps are dead
  // then), so Wd extends past the f temps if they need more room.
  MechDev &d = m.dev;
  d.S = S;
  d.R = R;
  d.max_reac = m.max_reac;
  d.n_phot = m.n_phot;
  d.n_pairs = n_pairs;
  d.d_Y = 0;
  d.d_ONE = S;
  d.d_ZERO = S + 1;
  std::vector<std::vector<std::pair<double, int>>> f_by_species(S);
  for (int j = 0; j < R; ++j)
    for (auto &kv : nu[j]) f_by_species[kv.first].push_back({kv.second, j});
  ConstTable fct;                          // the f program's constants, numbered before k~
  fct.base = S + 2;
  for (int i = 0; i < S; ++i)
    for (auto &t : f_by_species[i]) fct.get(t.first);
  d.d_KT = fct.base + (int)fct.vals.size();
  d.d_RT = d.d_KT + R;
  d.d_F = d.d_RT + R;
  int d_temp = d.d_F + S;
  // WL (LU precision): LU[nnz] (-1/u_kk in the pivot slots once factored),
  // ZERO, ONE, M temps, nu constants, solve temporaries.  The M program names the
  // pair products by the virtual indices P_VIRTUAL + pair, the solve programs the
  // solve vector by X_VIRTUAL + position (above every WL slot); their device
  // forms map them to Wd: the pair products to the rate and f slots (dead while M
  // is formed), the solve vector to y's slots (dead during a solve: y is written
  // before every f evaluation and formation of M).
  d.L_LU = 0;
  d.nnz_lu = nnz;
  d.L_X = X_VIRTUAL;
  d.L_P = P_VIRTUAL;
  d.L_ZERO = nnz;
  const int L_ONE = d.L_ZERO + 1;
  const int L_NEG_ONE = L_ONE + 1;
  int L_temp = L_NEG_ONE + 1;
  d.m_clear = nnz;

  // ---- f program: f_i = sum_j nu_ij r_j, species-major, chunked
  {
    const std::vector<std::vector<std::pair<double, int>>> &by_species = f_by_species;
    int n_temp = 0;
    for (int i = 0; i < S; ++i) n_temp += (int)std::max<size_t>(1, (by_species[i].size() + CHUNK - 1) / CHUNK) - 1;
    ConstTable &ct = fct;
    std::vector<std::vector<std::pair<int, int>>> terms(S);
    double flops = 0;
    for (int i = 0; i < S; ++i)
      for (auto &t : by_species[i]) {
        terms[i].push_back({ct.get(t.first), d.d_RT + t.second});
        flops += 2;
      }
    for (int j = 0; j < R; ++j) flops += rx[j].n_reac;
    Scheduler sch(d_temp + n_temp + 8);
    int temp_next = d_temp;
    for (int i = 0; i < S; ++i) add_sum(sch, d.d_F + i, true, terms[i], CHUNK, temp_next, d.d_ZERO, d.d_ONE);
    m.f_prog = sch.finish(true);
    m.flops_f = flops;
    d.Wd_len = std::max(d_temp + n_temp, d.d_RT + n_pairs);   // the pair products' slots (8 bytes at most)
    m.d_consts_v = {1.0, 0.0};
    m.d_consts_i = {d.d_ONE, d.d_ZERO};
    for (size_t k = 0; k < ct.vals.size(); ++k) {
      m.d_consts_v.push_back(ct.vals[k]);
      m.d_consts_i.push_back(ct.base + (int)k);
    }
  }

  // ---- pairs (reaction, reactant slot) and the M program
  {
    m.pair_rx.clear();
    m.pair_other.clear();
    std::vector<std::vector<std::pair<double, int>>> slot_terms(nnz);
    int pidx = 0;
    double flops = 0;
    for (int j = 0; j < R; ++j)
      for (int s = 0; s < rx[j].n_reac; ++s) {
        int o[2] = {d.d_ONE, d.d_ONE};
        int no = 0;
        for (int s2 = 0; s2 < rx[j].n_reac; ++s2)
          if (s2 != s) o[no++] = d.d_Y + rx[j].reac[s2];
        m.pair_rx.push_back(j);
        m.pair_other.push_back({o[0], o[1]});
        flops += rx[j].n_reac;    // k~ times the other reactants, times -c
        const int l = rx[j].reac[s];
        for (auto &kv : nu[j]) {
          const int sl = slot[m.pos[kv.first] * S + m.pos[l]];
          slot_terms[sl].push_back({kv.second, pidx});
        }
        pidx++;
      }
    int n_temp = 0;
    for (int k = 0; k < nnz; ++k)
      n_temp += (int)std::max<size_t>(1, (slot_terms[k].size() + CHUNK - 1) / CHUNK) - 1;
    ConstTable ct;
    ct.base = L_temp + n_temp;
    std::vector<std::vector<std::pair<int, int>>> terms(nnz);
    for (int k = 0; k < nnz; ++k)
      for (auto &t : slot_terms[k]) {
        terms[k].push_back({ct.get(t.first), d.L_P + t.second});
        flops += 2;
      }
    Scheduler sch(std::max(ct.base + (int)ct.vals.size() + 64, P_VIRTUAL + n_pairs + 1));
    int temp_next = L_temp;
    for (int k = 0; k < nnz; ++k)
      if (!terms[k].empty()) add_sum(sch, d.L_LU + k, false, terms[k], CHUNK, temp_next, d.L_ZERO, L_ONE);
    m.m_prog = sch.finish(true);
    m.flops_jac = flops;
    d.WL_len = ct.base + (int)ct.vals.size();
    m.L_consts_v = {0.0, 1.0, -1.0};
    m.L_consts_i = {d.L_ZERO, L_ONE, L_NEG_ONE};
    for (size_t k = 0; k < ct.vals.size(); ++k) {
      m.L_consts_v.push_back(ct.vals[k]);
      m.L_consts_i.push_back(ct.base + (int)k);
    }
  }

  // ---- LU program (right-looking, M = L D U'): L unit lower stored negated,
  // -1/u_kk in the pivot's own slot, U' unit upper stored negated (-u_kj/u_kk)
  {
    Scheduler sch(d.WL_len + 8);
    double flops = 0;
    m.lu_diag.assign(S, 0);
    for (int k = 0; k < S; ++k) m.lu_diag[k] = d.L_LU + slot[k * S + k];
    for (int k = 0; k < S; ++k) {
      const int dk = d.L_LU + slot[k * S + k];
      const int nk = dk;                // the reciprocal overwrites the pivot
      sch.recip(nk, dk);
      flops += 1;
      std::vector<int> Lc, Ur;
      for (int i = k + 1; i < S; ++i)
        if (F[i * S + k]) Lc.push_back(i);
      for (int j = k + 1; j < S; ++j)
        if (F[k * S + j]) Ur.push_back(j);
      for (int i : Lc) {
        const int ik = d.L_LU + slot[i * S + k];
        sch.fma(ik, ik, nk, d.L_ZERO);
        flops += 1;
      }
      for (int i : Lc)
        for (int j : Ur) {
          const int ij = d.L_LU + slot[i * S + j];
          sch.fma(ij, d.L_LU + slot[i * S + k], d.L_LU + slot[k * S + j], ij);
          flops += 2;
        }
      // U' = D^{-1} U: row k becomes -u_kj/u_kk once pivot k's updates have read it
      // (not counted: the factorisation's algorithmic flops are those of plain LU)
      for (int j : Ur) {
        const int kj = d.L_LU + slot[k * S + j];
        sch.fma(kj, kj, nk, d.L_ZERO);
      }
    }
    m.lu_prog = sch.finish(true);
    m.flops_lu = flops;
  }

  // ---- solves with the LDU factors, both programs without negation:
  // forward:  X = L^{-1} b, then X_k = ninv_k y_k = -(D^{-1} y)_k once every row
  //           that reads y_k has;
  // backward: V = -x from V_k = X_k + sum_{j>k} (-u'_kj) V_j (unit upper),
  // so the solution is -X.  Row-oriented, see emit_rows.
  std::vector<int> rows_up(S), rows_down(S), xloc(S);
  for (int k = 0; k < S; ++k) {
    rows_up[k] = k;
    rows_down[k] = S - 1 - k;
    xloc[k] = d.L_X + k;
  }
  const int L_STMP = d.WL_len;
  d.WL_len += NSTMP;
  {
    Scheduler f(X_VIRTUAL + S + 8), b(X_VIRTUAL + S + 8);
    std::vector<std::vector<std::pair<int, int>>> lt(S), ut(S);
    double flops = 0;
    for (int i = 0; i < S; ++i)
      for (int k = 0; k < S; ++k) {
        if (k < i && F[i * S + k]) lt[i].push_back({d.L_LU + slot[i * S + k], k});
        if (k > i && F[i * S + k]) ut[i].push_back({d.L_LU + slot[i * S + k], k});
      }
    for (int i = 0; i < S; ++i) flops += 2.0 * (double)(lt[i].size() + ut[i].size()) + 1.0;
    int tnext = 0;
    emit_rows(f, rows_up, lt, xloc, L_STMP, NSTMP, tnext, d.L_ZERO, L_ONE);
    for (int k = 0; k < S; ++k) f.fma(d.L_X + k, d.L_LU + slot[k * S + k], d.L_X + k, d.L_ZERO);
    emit_rows(b, rows_down, ut, xloc, L_STMP, NSTMP, tnext, d.L_ZERO, L_ONE);
    m.fwd_prog = f.finish();
    m.bwd_prog = b.finish();
    m.flops_solve = flops;
  }
  d.d_DUMMY = d.Wd_len++;
  d.L_DUMMY = d.WL_len++;

  // ---- discrete adjoint: the walks' per-cell slice is the forward's Wd and WL
  // (where every forward program expects them, the M program's WL slots included),
  // then the adjoint's own arrays and the partials dr_j/dy_l (PP); its programs
  // address the slice from its start (element indices in doubles: the adjoint is
  // FP64).
  {
    d.a_MU = ((d.Wd_len + 1) & ~1) + d.WL_len;
    d.a_NM = d.a_MU + S;
    d.a_JTM = d.a_NM + R;
    d.a_G = d.a_JTM + S;
    int temp0 = d.a_G + R;
    // nu_j . mu for every reaction, and J^T mu for every species
    std::vector<std::vector<std::pair<double, int>>> nd_terms(R);   // (nu, species)
    for (int j = 0; j < R; ++j)
      for (auto &kv : nu[j]) nd_terms[j].push_back({kv.second, kv.first});
    std::vector<std::vector<std::pair<int, int>>> jt_terms(S);      // (pair, reaction)
    {
      int pidx = 0;
      for (int j = 0; j < R; ++j)
        for (int s2 = 0; s2 < rx[j].n_reac; ++s2) jt_terms[rx[j].reac[s2]].push_back({pidx++, j});
    }
    int n_temp = 0;
    for (int j = 0; j < R; ++j) n_temp += (int)std::max<size_t>(1, (nd_terms[j].size() + CHUNK - 1) / CHUNK) - 1;
    for (int l = 0; l < S; ++l) n_temp += (int)std::max<size_t>(1, (jt_terms[l].size() + CHUNK - 1) / CHUNK) - 1;
    ConstTable ct;
    ct.base = temp0 + n_temp;
    Scheduler a(ct.base + 64 + 2 * R);
    int temp_next = temp0;
    for (int j = 0; j < R; ++j) {
      std::vector<std::pair<int, int>> terms;
      for (auto &t : nd_terms[j]) terms.push_back({ct.get(t.first), d.a_MU + t.second});
      add_sum(a, d.a_NM + j, true, terms, CHUNK, temp_next, d.d_ZERO, d.d_ONE);
    }
    // the constants are all known now, so the slice's length up to PP
    const int wda_len = ct.base + (int)ct.vals.size();
    d.a_PP = wda_len;
    Scheduler b(d.a_PP + n_pairs + 1);
    for (int l = 0; l < S; ++l) {
      std::vector<std::pair<int, int>> terms;
      for (auto &t : jt_terms[l]) terms.push_back({d.a_PP + t.first, d.a_NM + t.second});
      add_sum(b, d.a_JTM + l, true, terms, CHUNK, temp_next, d.d_ZERO, d.d_ONE);
    }
    m.nudot_prog = a.finish(true);
    m.jt_prog = b.finish(true);
    d.Wda_len = wda_len;
    m.a_consts_v = ct.vals;
    m.a_consts_i.clear();
    for (size_t k = 0; k < ct.vals.size(); ++k) m.a_consts_i.push_back(ct.base + (int)k);
    if ((size_t)(d.a_PP + n_pairs) * sizeof(double) > 0xfff0 || (size_t)d.Wda_len * sizeof(double) > 0xfff0) {
      msg = "mechanism too large for the adjoint's 16-bit byte offsets";
      return CHEM_EINVAL;
    }
    // M^T = U'^T D L^T: W = U'^{-T} b (unit lower, coefficients -u'_kj), X_k =
    // ninv_k W_k = -(D^{-1} W)_k, then Q = -mu from Q_i = X_i + sum_{k>i} (-l_ki) Q_k
    // (unit upper); mu = -X.  Both programs without negation.
    Scheduler f(X_VIRTUAL + S + 8), g(X_VIRTUAL + S + 8);
    {
      std::vector<std::vector<std::pair<int, int>>> uT(S), lT(S);
      for (int k = 0; k < S; ++k)
        for (int j = 0; j < S; ++j) {
          if (j > k && F[k * S + j]) uT[j].push_back({d.L_LU + slot[k * S + j], k});
          if (j < k && F[k * S + j]) lT[j].push_back({d.L_LU + slot[k * S + j], k});
        }
      int tnext = 0;
      emit_rows(f, rows_up, uT, xloc, L_STMP, NSTMP, tnext, d.L_ZERO, L_ONE);
      for (int k = 0; k < S; ++k) f.fma(d.L_X + k, d.L_LU + slot[k * S + k], d.L_X + k, d.L_ZERO);
      emit_rows(g, rows_down, lT, xloc, L_STMP, NSTMP, tnext, d.L_ZERO, L_ONE);
    }
    m.fwdT_prog = f.finish();
    m.bwdT_prog = g.finish();
    // Algorithmic flops per corrector iteration walked by the adjoint: the
    // transposed solve (as many as the forward solve), the rates r_j and the
    // partials dr_j/dy_l (n_reac - 1 multiplications per pair), nu_j . g (a
    // multiply-add per stoichiometric term), J^T g (one per pair), the theta
    // update (3 per reaction) and the vector updates of lambda (6 per species).
    // The tangent: tangent rates s_j = k~ sum_s (prod_{s' != s} y) v_s + k~ r dtheta_j
    // (n_reac (n_reac - 1) + (n_reac - 1) + n_reac products and sums, then 4 for
    // the theta term and k~), the f program's sums (2 per stoichiometric term),
    // one solve and 6 per species.
    double nu_terms = 0, rates = 0, partials = 0, trates = 0;
    for (int j = 0; j < R; ++j) {
      const double nr = rx[j].n_reac;
      nu_terms += (double)nu[j].size();
      rates += nr;
      partials += nr * (nr - 1.0);
      trates += nr * (nr - 1.0) + (nr - 1.0) + (nr - 1.0) + 4.0;
    }
    m.flops_adj_iter = m.flops_solve + rates + partials + 2.0 * nu_terms + 2.0 * n_pairs + 3.0 * R + 6.0 * S;
    m.flops_tan_iter = trates + 2.0 * nu_terms + m.flops_solve + 6.0 * S;
  }
  if ((size_t)(((d.Wd_len + 1) & ~1) + d.WL_len) * sizeof(double) > 0xfff0 || d.WL_len >= X_VIRTUAL) {
    msg = "mechanism too large: the per-cell work arrays exceed the 16-bit byte offsets of the warp programs";
    return CHEM_EINVAL;
  }
  // ---- bank layout (see bank_permutation): the LU slots, then every pass's lanes
  {
    const int L_ONE = d.L_ZERO + 1;
    // weights: runs per formation of M (about 4.6 Newton solves per factorisation
    // on the 72/186 workload; the adjoint's transposed solves once per iteration walked)
    const std::vector<BankProg> bp = {{&m.m_prog, 1.0},   {&m.lu_prog, 1.0},   {&m.fwd_prog, 4.6},
                                      {&m.bwd_prog, 4.6}, {&m.fwdT_prog, 1.0}, {&m.bwdT_prog, 1.0}};
    // lanes for the slots as numbered, then the permutation for those lanes, then the lanes again
    for (const BankProg &b : bp) bank_lanes(*b.hp, d.L_DUMMY, d.L_ZERO, L_ONE);
    std::vector<int> perm(nnz);
    for (int e = 0; e < nnz; ++e) perm[e] = e;
    bank_permutation(bp, nnz, d.L_DUMMY, d.L_ZERO, L_ONE, std::min<long>(700L * nnz, 2000000L), perm);
    auto remap = [&](uint16_t &f) {
      if (f < nnz) f = (uint16_t)perm[f];
    };
    for (const BankProg &b : bp)
      for (Op &o : b.hp->ops) {
        if (o.t == OP_EMPTY) continue;
        if (o.t & OP_RECIP) {
          uint16_t t = (uint16_t)(o.t & 0x7fff);
          remap(t);
          o.t = (uint16_t)(t | OP_RECIP);
          remap(o.a);
        } else {
          remap(o.t);
          remap(o.a);
          remap(o.b);
          remap(o.c);
        }
      }
    for (int &x : m.lu_diag) x = d.L_LU + perm[x - d.L_LU];
    for (const BankProg &b : bp) bank_lanes(*b.hp, d.L_DUMMY, d.L_ZERO, L_ONE);
    bank_lanes(m.f_prog, d.d_DUMMY, d.d_ZERO, d.d_ONE);
  }
  m.rx_slot_idx.assign((size_t)R * 3, d.d_ONE);
  for (int j = 0; j < R; ++j)
    for (int s2 = 0; s2 < rx[j].n_reac; ++s2) m.rx_slot_idx[(size_t)j * 3 + s2] = d.d_Y + rx[j].reac[s2];
  return 0;
}

namespace {

template <typename T>
int put(Mechanism &m, const std::vector<T> &v, const T **dst, std::string &msg) {
  *dst = nullptr;
  if (v.empty()) return 0;
  void *p = nullptr;
  if (cudaMalloc(&p, v.size() * sizeof(T)) != cudaSuccess) { msg = "cudaMalloc failed for mechanism tables"; return CHEM_ENOMEM; }
  m.allocations.push_back(p);
  if (cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) { msg = "cudaMemcpy of mechanism tables failed"; return CHEM_ECUDA; }
  *dst = (const T *)p;
  return 0;
}

// Device form of a program: byte offsets (off(element index)), empty slots
// as FMAs into the dummy slot (in a pass with reciprocals: a reciprocal of one
// into it), RECIP ops marked by c == DEV_RECIP.
template <typename Off>
std::vector<ushort4> device_ops_at(const HostProgram &hp, Off off, int dummy, int zero, int one) {
  std::vector<ushort4> v(hp.ops.size());
  const int np = hp.n_pass();
  for (int p = 0; p < np; ++p) {
    bool recip = false;
    for (int l = 0; l < WARP; ++l) {
      const Op &o = hp.ops[(size_t)p * WARP + l];
      if (o.t != OP_EMPTY && (o.t & OP_RECIP)) recip = true;
    }
    for (int l = 0; l < WARP; ++l) {
      const Op &o = hp.ops[(size_t)p * WARP + l];
      ushort4 &d = v[(size_t)p * WARP + l];
      if (o.t == OP_EMPTY) {
        d = recip ? make_ushort4(off(dummy), off(one), 0, DEV_RECIP)
                  : make_ushort4(off(dummy), off(zero), off(zero), off(zero));
      } else if (o.t & OP_RECIP) {
        d = make_ushort4(off(o.t & 0x7fff), off(o.a), 0, DEV_RECIP);
      } else {
        d = make_ushort4(off(o.t), off(o.a), off(o.b), off(o.c));
      }
    }
  }
  return v;
}

// ... with byte offsets elem * index from the program's own array
std::vector<ushort4> device_ops(const HostProgram &hp, int elem, int dummy, int zero, int one) {
  return device_ops_at(hp, [elem](int e) { return (unsigned short)(e * elem); }, dummy, zero, one);
}

// polynomial coefficients (in eta) of R(eta)_{jm} = prod_{l<m} (l - j eta)/(l+1)
void r_poly(int j, int mm, double *c /* QMAX+1 */) {
  for (int p = 0; p <= QMAX; ++p) c[p] = 0.0;
  c[0] = 1.0;
  for (int l = 0; l < mm; ++l) {
    double n[QMAX + 1] = {0};
    for (int p = 0; p <= QMAX; ++p) {
      n[p] += c[p] * (double)l / (double)(l + 1);
      if (p + 1 <= QMAX) n[p + 1] += -c[p] * (double)j / (double)(l + 1);
    }
    for (int p = 0; p <= QMAX; ++p) c[p] = n[p];
  }
}

struct BlobWriter {
  std::vector<unsigned char> buf;
  template <typename T>
  int add(const std::vector<T> &v) {
    const int off = (int)buf.size();
    const size_t n = v.size() * sizeof(T);
    buf.resize(off + ((n + 15) & ~(size_t)15), 0);
    if (n) std::memcpy(buf.data() + off, v.data(), n);
    return off;
  }
};

}  // namespace

int upload_mechanism(Mechanism &m, std::string &msg) {
  MechDev &d = m.dev;
  const int R = m.R, S = m.S;
  cudaGetDevice(&m.device);
  std::vector<int> kind(R), nreac(R), phot(R);
  std::vector<double> A(R), Ea(R), B(R), J(R), ext((size_t)R * RX_EXT, 0.0);
  int ip = 0;
  for (int j = 0; j < R; ++j) {
    const chem_reaction &r = m.rx[j];
    kind[j] = r.kind;
    nreac[j] = r.n_reac;
    phot[j] = r.kind == CHEM_PHOTOLYSIS ? ip++ : -1;
    A[j] = r.A;
    Ea[j] = r.Ea_over_R;
    B[j] = r.B;
    J[j] = r.J;
    const double e[RX_EXT] = {r.A2, r.Ea2_over_R, r.B2, r.A3, r.Ea3_over_R, r.B3, r.Fc, r.N};
    for (int k = 0; k < RX_EXT; ++k) ext[(size_t)j * RX_EXT + k] = e[k];
  }
  std::vector<double> thr2(7 * GRID_N), thr3(7 * GRID_N), g(GRID_N), lim(16, 0.0);
  for (int p = 0; p < 7; ++p)
    for (int i = GRID_IMIN; i <= GRID_IMAX; ++i) {
      // The error estimate of order p+1 is ||v|| / (p+1) with ||v||^2 = (1/S) sum (v_i w_i)^2, and
      // its grid thresholds are 1/(bias 2^(i(p+1)/8)); the kernel compares the raw warp sum
      // sum (v_i w_i)^2 with the thresholds squared and multiplied by S (p+1)^2.
      const double sc = (double)S * (double)((p + 1) * (p + 1));
      thr2[p * GRID_N + i - GRID_IMIN] = sc / (2.0 * 2.0 * exp2((double)i * (double)(p + 1) / 4.0));
      thr3[p * GRID_N + i - GRID_IMIN] = sc / (3.0 * 3.0 * exp2((double)i * (double)(p + 1) / 4.0));
    }
  for (int i = GRID_IMIN; i <= GRID_IMAX; ++i) g[i - GRID_IMIN] = exp2((double)i / 8.0);
  for (int q = 0; q < 8; ++q) {
    lim[q] = (double)S * (double)((q + 1) * (q + 1));   // error test: ||d||^2 / (q+1)^2 <= 1
    const double tol = 0.1 * (double)(q + 1);             // corrector: ||delta||^2 <= (0.1 (q+1))^2
    lim[8 + q] = (double)S * (tol * tol);
  }

  // the staged blobs, one per LU precision (identical section offsets)
  for (int prec = 0; prec < 2; ++prec) {
    const int el = prec == 0 ? 8 : 4;     // bytes per WL element
    BlobWriter bw;
    TableOffsets t;
    t.f_ops = bw.add(device_ops(m.f_prog, 8, d.d_DUMMY, d.d_ZERO, d.d_ONE));
    t.f_runs = bw.add(m.f_prog.runs());
    // the M and solve programs run on the whole per-cell slice: WL slots after Wd
    // (rounded to an even length), the pair products in Wd from the rates' first
    // slot, the solve vector in y's slots
    const int wl_off = ((d.Wd_len + 1) & ~1) * 8, p_off = d.d_RT * 8, x_off = d.d_Y * 8;
    auto coff = [&](int e) {
      return (unsigned short)(e >= P_VIRTUAL   ? p_off + (e - P_VIRTUAL) * el
                              : e >= X_VIRTUAL ? x_off + (e - X_VIRTUAL) * el
                                               : wl_off + e * el);
    };
    const std::vector<ushort4> m_dev = device_ops_at(m.m_prog, coff, d.L_DUMMY, d.L_ZERO, d.L_ZERO + 1);
    t.fwd_ops = bw.add(device_ops_at(m.fwd_prog, coff, d.L_DUMMY, d.L_ZERO, d.L_ZERO + 1));
    t.bwd_ops = bw.add(device_ops_at(m.bwd_prog, coff, d.L_DUMMY, d.L_ZERO, d.L_ZERO + 1));
    std::vector<uint2> slots(R);
    for (int j = 0; j < R; ++j)
      slots[j] = make_uint2((unsigned)(m.rx_slot_idx[j * 3] * 8) | ((unsigned)(m.rx_slot_idx[j * 3 + 1] * 8) << 16),
                            (unsigned)(m.rx_slot_idx[j * 3 + 2] * 8));
    t.rx_slots = bw.add(slots);
    t.pair_rx = bw.add(m.pair_rx);
    std::vector<unsigned> po(m.pair_other.size());
    for (size_t k = 0; k < po.size(); ++k)
      po[k] = (unsigned)(m.pair_other[k].first * 8) | ((unsigned)(m.pair_other[k].second * 8) << 16);
    t.pair_other = bw.add(po);
    std::vector<int> diag(S);
    for (int k = 0; k < S; ++k) diag[k] = m.lu_diag[k] * el;
    t.lu_diag = bw.add(diag);
    t.staged = (int)bw.buf.size();         // the rest is read from global memory
    std::vector<int> doff(m.d_consts_i.size()), loff(m.L_consts_i.size());
    for (size_t k = 0; k < doff.size(); ++k) doff[k] = m.d_consts_i[k] * 8;
    for (size_t k = 0; k < loff.size(); ++k) loff[k] = m.L_consts_i[k] * el;
    t.dconst_off = bw.add(doff);
    t.dconst_val = bw.add(m.d_consts_v);
    t.Lconst_off = bw.add(loff);
    t.Lconst_val = bw.add(m.L_consts_v);
    t.thr2 = bw.add(thr2);
    t.thr3 = bw.add(thr3);
    t.g = bw.add(g);
    t.lim = bw.add(lim);
    t.bytes = (int)bw.buf.size();
    d.tab = t;
    int rc = put(m, bw.buf, &d.blob[prec], msg);
    if (!rc) rc = put(m, m_dev, &d.m_ops[prec], msg);
    if (!rc) rc = put(m, device_ops(m.lu_prog, el, d.L_DUMMY, d.L_ZERO, d.L_ZERO + 1), &d.lu_ops[prec], msg);
    if (!rc && prec == 0) rc = put(m, m.m_prog.runs(), &d.m_runs, msg);
    if (!rc && prec == 0) rc = put(m, m.lu_prog.runs(), &d.lu_runs, msg);
    if (rc) {
      free_mechanism(m);
      return rc;
    }
  }
  {
    int rc = 0;
    // the transposed solves (FP64) on the whole per-cell slice, like the forward solves
    const int wl_off = ((d.Wd_len + 1) & ~1) * 8, x_off = d.d_Y * 8;
    auto xoff64 = [&](int e) { return (unsigned short)(e >= X_VIRTUAL ? x_off + (e - X_VIRTUAL) * 8 : wl_off + e * 8); };
    std::vector<int> aoff(m.a_consts_i.size());
    for (size_t k = 0; k < aoff.size(); ++k) aoff[k] = m.a_consts_i[k] * 8;
    if ((rc = put(m, aoff, &d.a_const_off, msg)) || (rc = put(m, m.a_consts_v, &d.a_const_val, msg)) ||
        (rc = put(m, device_ops(m.nudot_prog, 8, d.d_DUMMY, d.d_ZERO, d.d_ONE), &d.nudot_ops, msg)) ||
        (rc = put(m, device_ops(m.jt_prog, 8, d.d_DUMMY, d.d_ZERO, d.d_ONE), &d.jt_ops, msg)) ||
        (rc = put(m, device_ops_at(m.fwdT_prog, xoff64, d.L_DUMMY, d.L_ZERO, d.L_ZERO + 1), &d.fwdT_ops, msg)) ||
        (rc = put(m, device_ops_at(m.bwdT_prog, xoff64, d.L_DUMMY, d.L_ZERO, d.L_ZERO + 1), &d.bwdT_ops, msg)) ||
        (rc = put(m, m.nudot_prog.runs(), &d.nudot_runs, msg)) || (rc = put(m, m.jt_prog.runs(), &d.jt_runs, msg)) ||
        (rc = put(m, m.fwdT_prog.runs(), &d.fwdT_runs, msg)) || (rc = put(m, m.bwdT_prog.runs(), &d.bwdT_runs, msg))) {
      free_mechanism(m);
      return rc;
    }
    d.a_nconst = (int)m.a_consts_v.size();
    d.nudot_npass = m.nudot_prog.n_pass();
    d.jt_npass = m.jt_prog.n_pass();
    d.fwdT_npass = m.fwdT_prog.n_pass();
    d.bwdT_npass = m.bwdT_prog.n_pass();
    d.nudot_nruns = (int)m.nudot_prog.runs().size();
    d.jt_nruns = (int)m.jt_prog.runs().size();
    d.fwdT_nruns = (int)m.fwdT_prog.runs().size();
    d.bwdT_nruns = (int)m.bwdT_prog.runs().size();
  }
  d.f_npass = m.f_prog.n_pass();
  d.f_nruns = (int)m.f_prog.runs().size();
  d.m_nruns = (int)m.m_prog.runs().size();
  d.lu_nruns = (int)m.lu_prog.runs().size();
  d.fwd_npass = m.fwd_prog.n_pass();
  d.bwd_npass = m.bwd_prog.n_pass();
  d.m_npass = m.m_prog.n_pass();
  d.lu_npass = m.lu_prog.n_pass();
  d.d_nconst = (int)m.d_consts_v.size();
  d.L_nconst = (int)m.L_consts_v.size();

  // T(eta) = U R(eta), U = R(1): coefficients of each entry as a polynomial in eta
  std::vector<double> coef(QMAX * QMAX * (QMAX + 1), 0.0);
  for (int i = 1; i <= QMAX; ++i)
    for (int mm = 1; mm <= QMAX; ++mm) {
      double *acc = &coef[((i - 1) * QMAX + (mm - 1)) * (QMAX + 1)];
      for (int j = 1; j <= QMAX; ++j) {
        double u[QMAX + 1], r[QMAX + 1];
        r_poly(i, j, u);          // U_{ij} = R(1)_{ij}: the polynomial at eta = 1
        double uij = 0.0;
        for (int p = 0; p <= QMAX; ++p) uij += u[p];
        r_poly(j, mm, r);
        for (int p = 0; p <= QMAX; ++p) acc[p] += uij * r[p];
      }
    }
  int rc = 0;
  if ((rc = put(m, kind, &d.rx_kind, msg)) || (rc = put(m, nreac, &d.rx_nreac, msg)) ||
      (rc = put(m, phot, &d.rx_phot, msg)) || (rc = put(m, A, &d.rx_A, msg)) ||
      (rc = put(m, Ea, &d.rx_Ea, msg)) || (rc = put(m, B, &d.rx_B, msg)) || (rc = put(m, J, &d.rx_J, msg)) ||
      (rc = put(m, ext, &d.rx_ext, msg)) ||
      (rc = put(m, m.pos, &d.sp_pos, msg)) || (rc = put(m, coef, &d.rescale_coef, msg))) {
    free_mechanism(m);
    return rc;
  }
  {
    // reaction data of the derivative-design comparison: the records as given
    // (array of structures) and the same as separate arrays
    std::vector<int> reac((size_t)R * CHEM_MAX_REAC, 0), nprod(R), prod((size_t)R * CHEM_MAX_PROD, 0);
    std::vector<double> yld((size_t)R * CHEM_MAX_PROD, 0.0);
    for (int j = 0; j < R; ++j) {
      const chem_reaction &r = m.rx[j];
      for (int s = 0; s < r.n_reac; ++s) reac[(size_t)j * CHEM_MAX_REAC + s] = r.reac[s];
      nprod[j] = r.n_prod;
      for (int q = 0; q < r.n_prod; ++q) {
        prod[(size_t)j * CHEM_MAX_PROD + q] = r.prod[q];
        yld[(size_t)j * CHEM_MAX_PROD + q] = r.yield[q];
      }
    }
    if ((rc = put(m, m.rx, &d.rx_aos, msg)) || (rc = put(m, reac, &d.rx_reac, msg)) ||
        (rc = put(m, nprod, &d.rx_nprod, msg)) || (rc = put(m, prod, &d.rx_prod, msg)) ||
        (rc = put(m, yld, &d.rx_yld, msg))) {
      free_mechanism(m);
      return rc;
    }
  }
  if (set_constants() != cudaSuccess) {
    free_mechanism(m);
    msg = "could not set solver constants on the device";
    return CHEM_ECUDA;
  }
  return 0;
}

void free_mechanism(Mechanism &m) {
  for (void *p : m.allocations) cudaFree(p);
  m.allocations.clear();
}

}  // namespace chemgpu
