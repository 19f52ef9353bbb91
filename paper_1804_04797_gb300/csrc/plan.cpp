// Host planner: gate list -> passes over gathered tiles -> register/fused stages.
//
// Dependencies follow from two facts of the gate set (§2): one-qubit gates on
// different qubits commute, and diagonal gates (T, CZ, Z, projectors) commute with
// each other -- the property the paper's gate-scheduling preprocessor exploits (§2.3,
// "utilizes the diagonal properties of gate T and CZ").  A diagonal gate therefore
// never needs its qubits inside the tile: on a tile the non-tile qubits are fixed, so
// it becomes a conditional phase.  Only non-diagonal gates need their qubit in the
// tile, and the planner picks the tile qubits of each pass greedily to apply as many
// of them as the dependencies allow.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace svp {

void kind_matrix(int kind, double m[8]) {
  const double r = 1.0 / std::sqrt(2.0);
  const double c8 = std::cos(M_PI / 4), s8 = std::sin(M_PI / 4);
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // a, b, c, d as (re, im)
  switch (kind) {
    case K_H: v[0] = r; v[2] = r; v[4] = r; v[6] = -r; break;
    case K_T: v[0] = 1; v[6] = c8; v[7] = s8; break;
    case K_TDG: v[0] = 1; v[6] = c8; v[7] = -s8; break;
    case K_SX: v[0] = .5; v[1] = .5; v[2] = .5; v[3] = -.5; v[4] = .5; v[5] = -.5; v[6] = .5; v[7] = .5; break;
    case K_SXDG: v[0] = .5; v[1] = -.5; v[2] = .5; v[3] = .5; v[4] = .5; v[5] = .5; v[6] = .5; v[7] = -.5; break;
    case K_SY: v[0] = .5; v[1] = .5; v[2] = -.5; v[3] = -.5; v[4] = .5; v[5] = .5; v[6] = .5; v[7] = .5; break;
    case K_SYDG: v[0] = .5; v[1] = -.5; v[2] = .5; v[3] = -.5; v[4] = -.5; v[5] = .5; v[6] = .5; v[7] = -.5; break;
    case K_Z: v[0] = 1; v[6] = -1; break;
    case K_P0: v[0] = 1; break;
    case K_P1: v[6] = 1; break;
    default: v[0] = 1; v[6] = 1; break;
  }
  std::memcpy(m, v, sizeof(v));
}

namespace {

inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Which of the remaining gates a pass with tile qubit set S can apply, in list order.
// nd_block[q]: an earlier gate on q was deferred (blocks later non-diagonal gates on q).
// d_block[q]: an earlier NON-diagonal gate on q was deferred (blocks diagonal gates too;
// deferred diagonal gates commute with later diagonal ones).
struct Trial {
  int nondiag = 0, total = 0;
};

Trial run_trial(const std::vector<Gate> &g, const std::vector<int> &rem, uint64_t S,
                std::vector<char> *applied) {
  uint64_t nd_block = 0, d_block = 0;
  Trial t;
  if (applied) applied->assign(rem.size(), 0);
  for (size_t i = 0; i < rem.size(); ++i) {
    const Gate &x = g[rem[i]];
    const uint64_t qm = (1ull << x.q0) | (kind_two_qubit(x.kind) ? (1ull << x.q1) : 0ull);
    if (kind_is_diag(x.kind)) {
      if (qm & d_block) {
        nd_block |= qm;
      } else {
        ++t.total;
        if (applied) (*applied)[i] = 1;
      }
    } else {
      if ((qm & S) && !(qm & nd_block)) {
        ++t.total;
        ++t.nondiag;
        if (applied) (*applied)[i] = 1;
      } else {
        nd_block |= qm;
        d_block |= qm;
      }
    }
  }
  return t;
}

uint64_t choose_tile(int n, int m, int c, const std::vector<Gate> &g, const std::vector<int> &rem) {
  uint64_t S = (c >= 64) ? ~0ull : ((1ull << c) - 1);
  if (m >= n) return (n >= 64) ? ~0ull : ((1ull << n) - 1);
  // position of the first pending non-diagonal gate of each qubit (tie-breaker)
  std::vector<int> first(n, 1 << 30);
  for (size_t i = 0; i < rem.size(); ++i) {
    const Gate &x = g[rem[i]];
    if (!kind_is_diag(x.kind) && first[x.q0] == (1 << 30)) first[x.q0] = (int)i;
  }
  while (popc64(S) < m) {
    int best = -1;
    long long best_score = -1;
    for (int q = 0; q < n; ++q) {
      if (S & (1ull << q)) continue;
      Trial t = run_trial(g, rem, S | (1ull << q), nullptr);
      long long score = (long long)t.nondiag * (1ll << 40) + (long long)t.total * (1ll << 20) +
                        ((1 << 20) - 1 - std::min(first[q], (1 << 20) - 1));
      if (score > best_score) { best_score = score; best = q; }
    }
    S |= 1ull << best;
  }
  return S;
}

// Order of residues used by the tile's shared-memory swizzle: local bit p toggles
// bank-slot bit (p mod 4).  Lane bits with distinct residues make a half-warp's
// 8-byte accesses conflict-free.
void order_group_bits(int m, const std::vector<int> &nonr, uint8_t *out) {
  std::vector<int> lanes, rest;
  bool used_res[4] = {false, false, false, false};
  for (int b : nonr) {
    if ((int)lanes.size() < 4 && !used_res[b & 3]) { used_res[b & 3] = true; lanes.push_back(b); }
    else rest.push_back(b);
  }
  std::vector<int> all = lanes;
  for (int b : rest) all.push_back(b);
  (void)m;
  for (size_t i = 0; i < all.size(); ++i) out[i] = (uint8_t)all[i];
}

// Packed tiles: pair index k (tile bits 1..m-1) is stored at 16-byte slot pack_phys(k,
// layout).  Layout 0: pair bit i toggles slot bit (i mod 3).  Layout 1 (the TMA 128-byte
// swizzle): tile bits 1..3 toggle slot bits 0..2 directly, tile bits 4..6 (a box's row)
// toggle them too, higher tile bits none.  A quarter warp (8 lanes, one 128-byte wavefront
// of 16-byte accesses) is conflict-free when its three lane bits toggle three independent
// bank-group bit patterns.
uint32_t pack_offset(int tile_bit, int layout) { return 16u * pack_phys(1u << (tile_bit - 1), layout); }

// The bank-group bits (16-byte slot bits 0..2) a tile bit toggles.
uint32_t bank_bits(int tile_bit, int layout) { return pack_phys(1u << (tile_bit - 1), layout) & 7u; }

// Order the stage's group bits with three conflict-free lane bits first.  Layout 1, last
// stage of a pass: tile bits 1..3 go first when all three are group bits, so that a
// quarter warp's 16-byte stores of the last stage (straight from registers to HBM) fill
// one 128-byte line.
void order_group_bits_packed(const std::vector<int> &nonr, uint8_t *out, int layout, bool last_stage) {
  std::vector<int> lanes, rest;
  std::vector<int> cand = nonr;
  if (layout == 1) {
    // low tile bits first (coalesced stores), then the box rows, then the rest
    std::stable_sort(cand.begin(), cand.end(), [](int a, int b) { return a < b; });
    const bool low3 = std::count(nonr.begin(), nonr.end(), 1) && std::count(nonr.begin(), nonr.end(), 2) &&
                      std::count(nonr.begin(), nonr.end(), 3);
    if (last_stage && low3) {
      lanes = {1, 2, 3};
      for (int b : cand)
        if (b > 3) rest.push_back(b);
    }
  }
  if (lanes.empty()) {
    uint32_t span = 0;  // bank-group patterns covered so far (unit vectors in both layouts)
    for (int b : cand) {
      const uint32_t v = layout == 1 ? bank_bits(b, layout) : (1u << ((b - 1) % 3));
      if ((int)lanes.size() < 3 && v && !(span & v)) { span |= v; lanes.push_back(b); }
      else rest.push_back(b);
    }
  }
  std::vector<int> all = lanes;
  for (int b : rest) all.push_back(b);
  for (size_t i = 0; i < all.size(); ++i) out[i] = (uint8_t)all[i];
}

}  // namespace

bool build_plan(int n, const std::vector<Gate> &gates, const Options &opt, bool fresh_state,
                Plan *plan, const char **err) {
  Plan &P = *plan;
  P = Plan();
  P.n = n;
  P.layout = opt.layout;
  const int m = std::min(opt.m, n);
  const int c = std::min(opt.c, m);
  const bool pack = opt.pack;
  // packed: tile bit 0 is in every stage, besides up to rk register slots
  const int rk = std::min(opt.rk, pack ? m - 1 : m);
  const int r = std::min(std::min(opt.r, rk), m);
  if (m > kMaxTileBits || rk > kMaxReg || r < 1 || c < 0 || m - rk > 12) { *err = "bad tile shape"; return false; }
  P.rk = rk;
  if (pack && (rk < 1 || m < rk + 1 || c < 1)) { *err = "packed plan needs tiles of >= rk + 1 qubits"; return false; }
  if (opt.layout == 1 && (!pack || c != 4 || m < 7 || m > 13)) { *err = "TMA tile layout needs packed tiles of 7..13 qubits with 4 low ones"; return false; }

  // leading layer of H on every qubit of a fresh state -> uniform first pass
  size_t start = 0;
  if (fresh_state) {
    uint64_t seen = 0;
    size_t i = 0;
    while (i < gates.size() && gates[i].kind == K_H && !(seen & (1ull << gates[i].q0))) {
      seen |= 1ull << gates[i].q0;
      ++i;
      if (popc64(seen) == n) break;
    }
    if (popc64(seen) == n) { start = i; P.init_uniform = true; }
  }
  for (size_t i = 0; i < start; ++i) { P.order.push_back((int)i); P.pass_of.push_back(0); }

  std::vector<int> rem;
  for (size_t i = start; i < gates.size(); ++i) rem.push_back((int)i);

  // Gate scheduling that uses the diagonal T and CZ (§2.3), one step further for T.  Plans
  // for the plain pipelined kernels: a T (or its adjoint) on a qubit of the tile
  // waits for the next non-diagonal gate on its qubit (succ) and is placed in the same
  // pass and stage, right before it in the stage's ops, where the kernel applies both as
  // one step (its factor 1/sqrt2 rides on the gate's fused operations).  A phase commutes
  // with every gate between the two (diagonal gates on its qubit, any gate on others).
  // (34 qubits, fixed kernel shapes: 0.381 s -> 0.371 s, pass 0 64 -> 57 ms.  Deferring
  // also the phases on qubits outside the tile, which the pass applies as a scalar phase
  // of the tile, measured the same with a larger norm drift.)
  const bool lazy = pack && !opt.fused && opt.layout == 1;
  std::vector<int> succ(gates.size(), -1);
  if (lazy) {
    std::vector<int> next_nd(n, -1);
    for (size_t i = gates.size(); i-- > start;) {
      const Gate &x = gates[i];
      if (x.kind == K_T || x.kind == K_TDG) succ[i] = next_nd[x.q0];
      if (!kind_is_diag(x.kind)) next_nd[x.q0] = (int)i;
    }
  }
  auto lazy_phase = [&](int gi) { return lazy && succ[(size_t)gi] >= 0; };

  const double amps = std::ldexp(1.0, n);
  bool first_pass = true;
  // packed plans: the square roots' scalars not yet applied -- an odd factor 2^{-1/2}
  // carried between stages, and the phase e^{i pi phase8/4} -- for the plan's end
  int sqrt_carry = 0, phase8 = 0;
  while (!rem.empty() || (first_pass && fresh_state)) {
    const uint64_t S = choose_tile(n, m, c, gates, rem);
    std::vector<char> applied;
    run_trial(gates, rem, S, &applied);
    if (lazy) {
      // a waiting phase on a tile qubit goes to the pass of its successor
      std::vector<char> app(gates.size(), 0), keep = applied;
      for (size_t i = 0; i < rem.size(); ++i) app[(size_t)rem[i]] = applied[i];
      bool any = false;
      for (size_t i = 0; i < rem.size(); ++i) {
        const Gate &x = gates[rem[i]];
        if (applied[i] && lazy_phase(rem[i]) && ((S >> x.q0) & 1ull) && !app[(size_t)succ[(size_t)rem[i]]])
          applied[i] = 0;
        any = any || applied[i];
      }
      if (!any) applied = keep;  // (never: the tile holds a pending non-diagonal gate)
      // phases on qubits outside the tile cost one scalar phase of the tile per stage
      // (complex products on every amplitude): a pass with only one or two of them, and no
      // other, sends them on to the passes of their successors instead (34 qubits: pass 4
      // 48.7 -> 47.7 ms, its one such phase now rides on a gate in pass 5)
      int n_t = 0, n_other = 0;
      for (size_t i = 0; i < rem.size(); ++i) {
        const Gate &x = gates[rem[i]];
        if (!applied[i] || !kind_is_diag(x.kind)) continue;
        const bool out0 = !((S >> x.q0) & 1ull), out1 = kind_two_qubit(x.kind) ? !((S >> x.q1) & 1ull) : true;
        if (!out0 || !out1) continue;
        (lazy_phase(rem[i]) ? n_t : n_other) += 1;
      }
      if (n_other == 0 && n_t > 0 && n_t <= 2) {
        std::vector<char> fewer = applied;
        bool left_any = false;
        for (size_t i = 0; i < rem.size(); ++i) {
          if (fewer[i] && lazy_phase(rem[i]) && !((S >> gates[rem[i]].q0) & 1ull)) fewer[i] = 0;
          left_any = left_any || fewer[i];
        }
        if (left_any) applied = fewer;
      }
    }
    if (lazy && first_pass && fresh_state) {
      // The write-only first pass is bound by its arithmetic, the passes after it by HBM:
      // on each qubit that this tile shares with the next pass's, the last non-diagonal
      // gate (with the T waiting for it and the diagonal gates after it) moves to the next
      // pass when nothing else here depends on it and the next tile stays the same.
      std::vector<int> rest;
      for (size_t i = 0; i < rem.size(); ++i)
        if (!applied[i]) rest.push_back(rem[i]);
      const uint64_t S1 = choose_tile(n, m, c, gates, rest);
      std::vector<char> moved = applied;
      // position in rem of the last applied non-diagonal gate of each qubit (-1: none)
      std::vector<int> last_nd(n, -1);
      for (size_t i = 0; i < rem.size(); ++i)
        if (moved[i] && !kind_is_diag(gates[rem[i]].kind)) last_nd[gates[rem[i]].q0] = (int)i;
      for (int q = 0; q < n; ++q) {
        if (!((S >> q) & 1ull) || !((S1 >> q) & 1ull)) continue;
        const int last = last_nd[q];
        if (last < 0) continue;
        // what follows it on q here must be diagonal, and a CZ among it must have no
        // applied non-diagonal gate after it on its other qubit
        bool ok = true;
        std::vector<size_t> with;
        for (size_t i = (size_t)last + 1; i < rem.size() && ok; ++i) {
          if (!moved[i]) continue;
          const Gate &x = gates[rem[i]];
          const bool on_q = x.q0 == q || (kind_two_qubit(x.kind) && x.q1 == q);
          if (!on_q) continue;
          if (!kind_is_diag(x.kind)) { ok = false; break; }
          if (kind_two_qubit(x.kind) && last_nd[x.q0 == q ? x.q1 : x.q0] > (int)i) { ok = false; break; }
          with.push_back(i);
        }
        if (!ok) continue;
        moved[(size_t)last] = 0;
        last_nd[q] = -1;
        for (int i = last - 1; i >= 0; --i)
          if (moved[(size_t)i] && !kind_is_diag(gates[rem[(size_t)i]].kind) && gates[rem[(size_t)i]].q0 == q) {
            last_nd[q] = i;
            break;
          }
        for (size_t i : with) moved[i] = 0;
        for (size_t i = 0; i < rem.size(); ++i)  // the T that waits for it
          if (moved[i] && lazy_phase(rem[i]) && succ[(size_t)rem[i]] == rem[(size_t)last]) moved[i] = 0;
      }
      std::vector<int> rest2;
      bool left_any = false;
      for (size_t i = 0; i < rem.size(); ++i) {
        if (!moved[i]) rest2.push_back(rem[i]);
        left_any = left_any || moved[i];
      }
      if (left_any && moved != applied && choose_tile(n, m, c, gates, rest2) == S1) applied = moved;
    }
    std::vector<int> now, later;
    for (size_t i = 0; i < rem.size(); ++i) (applied[i] ? now : later).push_back(rem[i]);
    std::vector<int> pos_in_now;  // gate index -> position in `now` (-1: not in this pass)
    if (lazy) {
      pos_in_now.assign(gates.size(), -1);
      for (size_t i = 0; i < now.size(); ++i) pos_in_now[(size_t)now[i]] = (int)i;
    }

    DevPass dp;
    std::memset(&dp, 0, sizeof(dp));
    dp.m = (uint8_t)m;
    dp.c = (uint8_t)c;
    dp.n = (uint8_t)n;
    int local_of[64];
    for (int q = 0; q < 64; ++q) local_of[q] = -1;
    {
      // Layout 1: tile bits 4..6 are the rows of the 8-row TMA boxes, the only high tile
      // bits that toggle shared-memory bank groups.  They go to the three high tile qubits
      // with the fewest non-diagonal gates in the pass (seldom register qubits of a stage,
      // so they are free to serve as conflict-free lane bits); the rest follow ascending.
      std::vector<int> high;
      for (int q = c; q < n; ++q)
        if (S & (1ull << q)) high.push_back(q);
      if (opt.layout == 1 && high.size() >= 3) {
        std::vector<int> nd(n, 0);
        for (int gi : now)
          if (!kind_is_diag(gates[gi].kind)) ++nd[gates[gi].q0];
        std::vector<int> rows = high;
        std::stable_sort(rows.begin(), rows.end(), [&](int a, int b) { return nd[a] < nd[b]; });
        rows.resize(3);
        std::sort(rows.begin(), rows.end());
        std::vector<int> rest;
        for (int q : high)
          if (std::find(rows.begin(), rows.end(), q) == rows.end()) rest.push_back(q);
        high = rows;
        high.insert(high.end(), rest.begin(), rest.end());
      }
      int li = 0;
      for (int q = 0; q < c; ++q) { dp.tq[li] = (uint8_t)q; local_of[q] = li++; }
      for (int q : high) { dp.tq[li] = (uint8_t)q; local_of[q] = li++; }
      int ni = 0;
      for (int q = 0; q < n; ++q)
        if (!(S & (1ull << q))) dp.ntq[ni++] = (uint8_t)q;
      dp.nt = (uint8_t)ni;
    }
    if (pack) dp.flags |= PF_PACKED;
    if (first_pass && fresh_state) {
      dp.flags |= P.init_uniform ? PF_INIT_UNIFORM : PF_INIT_ZERO;
      dp.init_amp = P.init_uniform ? (float)std::pow(2.0, -0.5 * n) : 1.0f;
      P.hbm_bytes += 8.0 * amps;
    } else {
      P.hbm_bytes += 16.0 * amps;
    }
    dp.stage_begin = (uint32_t)P.stages.size();

    // ---- stages: groups of <= r register bits ------------------------------------
    std::vector<char> done(now.size(), 0);
    size_t left = now.size();
    // Schedule one stage with a fixed register set Rm (tile-local bit mask): non-diagonal
    // gates on register bits (not yet closed), diagonal gates inside Rm as inner gates,
    // other diagonal gates as post gates that close their tile bits for the rest of the
    // stage.  Marks the placed gates in dn; returns (non-diagonal placed, total placed).
    auto run_stage = [&](uint32_t Rm, std::vector<char> &dn, std::vector<int> *inner,
                         std::vector<int> *post) -> std::pair<int, int> {
      uint32_t closed = 0;
      int nd = 0, tot = 0;
      std::vector<size_t> here;  // positions placed by this call
      bool progress = true;
      while (progress) {
        progress = false;
        uint64_t pend_nd = 0, pend_any = 0;  // qubits with an earlier unscheduled gate
        for (size_t i = 0; i < now.size(); ++i) {
          if (dn[i]) continue;
          const Gate &x = gates[now[i]];
          const uint64_t qm = (1ull << x.q0) | (kind_two_qubit(x.kind) ? (1ull << x.q1) : 0ull);
          const bool diag = kind_is_diag(x.kind);
          // ready: no earlier unscheduled gate that fails to commute with this one
          const bool ready = diag ? !(qm & pend_nd) : !(qm & pend_any);
          bool placed = false;
          if (ready) {
            if (!diag) {
              const int a = local_of[x.q0];
              if (((Rm >> a) & 1u) && !((closed >> a) & 1u)) {
                if (inner) inner->push_back(now[i]);
                placed = true;
                ++nd;
              }
            } else {
              bool all_in = true;
              uint32_t locals = 0;
              const int qs[2] = {x.q0, x.q1};
              for (int t = 0; t < (kind_two_qubit(x.kind) ? 2 : 1); ++t) {
                const int a = local_of[qs[t]];
                if (a < 0) { all_in = false; continue; }
                locals |= 1u << a;
                if (!((Rm >> a) & 1u)) all_in = false;
              }
              // The tensor-core kernel applies the inner gates as one matrix, so a diagonal
              // gate on a qubit outside the register set must follow it (a post gate) and
              // closes its register qubits for the rest of the stage.  The plain kernels
              // apply it in place as a phase conditioned on the fixed qubit.
              if (all_in || !opt.fused) { if (inner) inner->push_back(now[i]); }
              else { if (post) post->push_back(now[i]); closed |= locals; }
              placed = true;
            }
          }
          if (placed) {
            dn[i] = 1;
            ++tot;
            progress = true;
            here.push_back(i);
          } else {
            pend_any |= qm;
            if (!diag) pend_nd |= qm;
          }
        }
      }
      if (lazy) {
        // a waiting phase stays in this stage only with its successor (nothing placed
        // here depends on it otherwise: the successor is the next non-commuting gate)
        for (size_t i : here) {
          if (!lazy_phase(now[i])) continue;
          const int ps = pos_in_now[(size_t)succ[(size_t)now[i]]];
          if (ps < 0 || dn[(size_t)ps]) continue;  // successor in a later pass, or placed too
          dn[i] = 0;
          --tot;
          if (inner) inner->erase(std::find(inner->begin(), inner->end(), now[i]));
        }
      }
      return {nd, tot};
    };
    // The register qubits of every stage, by the same greedy choice as below on copies of
    // the schedule (they do not depend on the tile's bit order).
    auto stage_register_qubits = [&]() {
      std::vector<uint64_t> sets;
      std::vector<char> dn = done;
      size_t lf = left;
      std::vector<int> by_qubit;
      for (int bb = 0; bb < m; ++bb) by_qubit.push_back(bb);
      std::sort(by_qubit.begin(), by_qubit.end(), [&](int a, int b) { return dp.tq[a] < dp.tq[b]; });
      while (lf > 0) {
        uint32_t Rm = pack ? 1u : 0u;
        std::pair<int, int> cur;
        {
          std::vector<char> tmp = dn;
          cur = run_stage(Rm, tmp, nullptr, nullptr);
        }
        for (int round = 0; round < r; ++round) {
          int best = -1;
          std::pair<int, int> bs = cur;
          for (int bb : by_qubit) {
            if ((Rm >> bb) & 1u) continue;
            std::vector<char> tmp = dn;
            const std::pair<int, int> sc = run_stage(Rm | (1u << bb), tmp, nullptr, nullptr);
            if (sc.first > bs.first || (sc.first == bs.first && sc.second > bs.second)) { bs = sc; best = bb; }
          }
          if (best < 0) break;
          Rm |= 1u << best;
          cur = bs;
        }
        const std::pair<int, int> placed = run_stage(Rm, dn, nullptr, nullptr);
        if (placed.second == 0) break;
        lf -= (size_t)placed.second;
        uint64_t q = 0;
        for (int bb = 1; bb < m; ++bb)
          if ((Rm >> bb) & 1u) q |= 1ull << dp.tq[bb];
        sets.push_back(q);
      }
      return sets;
    };
    // Layout 1: the three box rows (tile bits 4, 5, 6; bank groups like qubits 1, 2, 3) are
    // chosen so that the fewest stages lack a group (lane) qubit of some bank group: a stage
    // has one for group k unless both qubit k+1 and row k are among its register qubits.
    // Ties: the rows with the fewest non-diagonal gates (the order above).
    if (opt.layout == 1 && m - c >= 3 && c == 4) {
      const std::vector<uint64_t> regs = stage_register_qubits();
      std::vector<int> high(dp.tq + 4, dp.tq + m);  // current order: quietest rows first
      int best_miss = 1 << 30;
      int best[3] = {high[0], high[1], high[2]};
      for (size_t a = 0; a < high.size(); ++a)
        for (size_t b = 0; b < high.size(); ++b)
          for (size_t d = 0; d < high.size(); ++d) {
            if (a == b || a == d || b == d) continue;
            const int rows[3] = {high[a], high[b], high[d]};
            int miss = 0;
            for (uint64_t R : regs)
              for (int k = 0; k < 3; ++k)
                if (((R >> (k + 1)) & 1ull) && ((R >> rows[k]) & 1ull)) ++miss;
            if (miss < best_miss) {
              best_miss = miss;
              for (int k = 0; k < 3; ++k) best[k] = rows[k];
            }
          }
      std::vector<int> order(best, best + 3);
      for (int q : high)
        if (q != best[0] && q != best[1] && q != best[2]) order.push_back(q);
      for (int i = 0; i < m - c; ++i) {
        dp.tq[c + i] = (uint8_t)order[(size_t)i];
        local_of[order[(size_t)i]] = c + i;
      }
    }
    while (left > 0) {
      // register bits by greedy lookahead: add the tile bit that lets the stage place the
      // most non-diagonal gates (then the most gates), up to r bits
      uint32_t Rm = pack ? 1u : 0u;
      std::pair<int, int> cur;
      {
        std::vector<char> tmp = done;
        cur = run_stage(Rm, tmp, nullptr, nullptr);
      }
      // candidates in ascending global qubit (ties go to the lower qubit whatever the
      // tile's bit order, so a layout's reordering of the tile bits changes no stage)
      std::vector<int> by_qubit;
      for (int bb = 0; bb < m; ++bb) by_qubit.push_back(bb);
      std::sort(by_qubit.begin(), by_qubit.end(), [&](int a, int b) { return dp.tq[a] < dp.tq[b]; });
      for (int round = 0; round < r; ++round) {
        int best = -1;
        std::pair<int, int> bs = cur;
        for (int bb : by_qubit) {
          if ((Rm >> bb) & 1u) continue;
          std::vector<char> tmp = done;
          const std::pair<int, int> sc = run_stage(Rm | (1u << bb), tmp, nullptr, nullptr);
          if (sc.first > bs.first || (sc.first == bs.first && sc.second > bs.second)) { bs = sc; best = bb; }
        }
        if (best < 0) break;
        Rm |= 1u << best;
        cur = bs;
      }
      std::vector<int> inner, post;
      const std::pair<int, int> placed = run_stage(Rm, done, &inner, &post);
      if (placed.second == 0) { *err = "planner: a stage placed no gate"; return false; }
      left -= (size_t)placed.second;
      const bool last_stage = left == 0;
      std::vector<int> R;
      for (int bb = pack ? 1 : 0; bb < m; ++bb)
        if ((Rm >> bb) & 1u) R.push_back(bb);
      // device stage
      DevStage ds;
      std::memset(&ds, 0, sizeof(ds));
      ds.r = (uint8_t)R.size();
      // the kernel holds 2^rk amplitudes (packed: pairs) per thread: pad the register
      // bits with unused tile bits (the fused kernel uses the first r of them)
      std::vector<int> rb = R;
      const int rpad = rk;
      // layout 1: padding from the tile bits that toggle no bank group (7 and up) first,
      // so that the ones that do (1..6) stay group bits, free to be conflict-free lanes
      std::vector<int> pad_order;
      if (opt.layout == 1)
        for (int b = m - 1; b >= 1; --b) pad_order.push_back(b);
      else
        for (int b = pack ? 1 : 0; b < m; ++b) pad_order.push_back(b);
      for (int b : pad_order) {
        if ((int)rb.size() >= rpad) break;
        if (std::find(rb.begin(), rb.end(), b) == rb.end()) rb.push_back(b);
      }
      for (int j = 0; j < rpad; ++j) ds.rbit[j] = (uint8_t)rb[j];
      std::vector<int> nonr;
      for (int b = pack ? 1 : 0; b < m; ++b)
        if (std::find(rb.begin(), rb.end(), b) == rb.end()) nonr.push_back(b);
      if (pack) order_group_bits_packed(nonr, ds.nonr, opt.layout, last_stage);
      else order_group_bits(m, nonr, ds.nonr);
      const int group_bits = (int)nonr.size();
      for (int half = 0; half < kRegEntry / 16; ++half) {
        for (int v = 0; v < 16; ++v) {
          DevGroupEntry ge;
          std::memset(&ge, 0, sizeof(ge));
          for (int i = 0; i < 4; ++i) {
            const int gi = 4 * half + i;
            if (!((v >> i) & 1) || gi >= group_bits) continue;
            ge.L ^= pack ? pack_offset(ds.nonr[gi], opt.layout) : (1u << ds.nonr[gi]);
            ge.G |= 1ull << dp.tq[ds.nonr[gi]];
          }
          P.gtab.push_back(ge);
        }
      }
      for (int e = kRegEntry; e < kGroupEntries; ++e) {
        DevGroupEntry ge;
        std::memset(&ge, 0, sizeof(ge));
        const int j = e - kRegEntry;
        if (pack && j < rpad) {
          ge.L = pack_offset(rb[j], opt.layout);
          ge.G = 1ull << dp.tq[rb[j]];
        }
        P.gtab.push_back(ge);
      }
      ds.op_begin = (uint32_t)P.ops.size();
      ds.diag_only = inner.empty() ? 1 : 0;
      auto reg_of = [&](int q) -> int {
        const int a = local_of[q];
        if (a < 0) return -1;
        if (pack && a == 0) return kPackSlot;
        for (int j = 0; j < rpad; ++j)
          if (rb[j] == a) return j;
        return -1;
      };
      auto emit = [&](uint8_t act, int j, int k, int arg, uint64_t cm, uint64_t cv) {
        DevOp o;
        std::memset(&o, 0, sizeof(o));
        if ((act == A_CZ || act == A_PEQ) && j > k) std::swap(j, k);  // both symmetric
        o.act = act; o.j = (uint8_t)(j < 0 ? 0 : j); o.k = (uint8_t)(k < 0 ? 0 : k);
        o.arg = (uint8_t)arg; o.cmask = cm; o.cval = cv;
        if (pack) {
          switch (act) {
            case A_H: o.code = P_PAIR + 0 + o.j; break;
            case A_SX: o.code = P_PAIR + 6 + o.j; break;
            case A_SY: o.code = P_PAIR + 12 + o.j; break;
            case A_SXDG: o.code = P_PAIR + 18 + o.j; break;
            case A_SYDG: o.code = P_PAIR + 24 + o.j; break;
            case A_T: o.code = P_DIAG + 0 + o.j; break;
            case A_TDG: o.code = P_DIAG + 6 + o.j; break;
            case A_Z: o.code = P_DIAG + 12 + o.j; break;
            case A_P0: o.code = P_DIAG + 18 + o.j; break;
            case A_P1: o.code = P_DIAG + 24 + o.j; break;
            case A_CZ: o.code = P_CZ + 6 * o.j + o.k; break;
            case A_PEQ: o.code = P_PEQ + 6 * o.j + o.k; break;
            case A_PHASE: o.code = P_PHASE; break;
            case A_ZERO: o.code = P_ZERO; break;
            default: o.code = P_U + o.j; break;
          }
          P.ops.push_back(o);
          return;
        }
        switch (act) {
          case A_H: o.code = C_PAIR + 0 + o.j; break;
          case A_SX: o.code = C_PAIR + 5 + o.j; break;
          case A_SY: o.code = C_PAIR + 10 + o.j; break;
          case A_SXDG: o.code = C_PAIR + 15 + o.j; break;
          case A_SYDG: o.code = C_PAIR + 20 + o.j; break;
          case A_T: o.code = C_DIAG + 0 + o.j; break;
          case A_TDG: o.code = C_DIAG + 5 + o.j; break;
          case A_Z: o.code = C_DIAG + 10 + o.j; break;
          case A_P0: o.code = C_DIAG + 15 + o.j; break;
          case A_P1: o.code = C_DIAG + 20 + o.j; break;
          case A_CZ: o.code = C_CZ + 5 * o.j + o.k; break;
          case A_PEQ: o.code = C_PEQ + 5 * o.j + o.k; break;
          case A_PHASE: o.code = C_PHASE; break;
          case A_ZERO: o.code = C_ZERO; break;
          default: o.code = C_U + o.j; break;
        }
        P.ops.push_back(o);
      };
      auto lower = [&](int gi) {
        const Gate &x = gates[gi];
        const int j = reg_of(x.q0);
        const int k = kind_two_qubit(x.kind) ? reg_of(x.q1) : -1;
        const uint64_t b0 = 1ull << x.q0, b1 = 1ull << x.q1;
        switch (x.kind) {
          case K_H: emit(A_H, j, 0, 0, 0, 0); break;
          case K_SX: emit(A_SX, j, 0, 0, 0, 0); break;
          case K_SY: emit(A_SY, j, 0, 0, 0, 0); break;
          case K_SXDG: emit(A_SXDG, j, 0, 0, 0, 0); break;
          case K_SYDG: emit(A_SYDG, j, 0, 0, 0, 0); break;
          case K_T: if (j >= 0) emit(A_T, j, 0, 0, 0, 0); else emit(A_PHASE, 0, 0, 1, b0, b0); break;
          case K_TDG: if (j >= 0) emit(A_TDG, j, 0, 0, 0, 0); else emit(A_PHASE, 0, 0, 7, b0, b0); break;
          case K_Z: if (j >= 0) emit(A_Z, j, 0, 0, 0, 0); else emit(A_PHASE, 0, 0, 4, b0, b0); break;
          case K_P0: if (j >= 0) emit(A_P0, j, 0, 0, 0, 0); else emit(A_ZERO, 0, 0, 0, b0, b0); break;
          case K_P1: if (j >= 0) emit(A_P1, j, 0, 0, 0, 0); else emit(A_ZERO, 0, 0, 0, b0, 0); break;
          case K_CZ:
            if (j >= 0 && k >= 0) emit(A_CZ, j, k, 0, 0, 0);
            else if (j >= 0) emit(A_Z, j, 0, 0, b1, b1);
            else if (k >= 0) emit(A_Z, k, 0, 0, b0, b0);
            else emit(A_PHASE, 0, 0, 4, b0 | b1, b0 | b1);
            break;
          case K_PEQ:
            if (j >= 0 && k >= 0) emit(A_PEQ, j, k, 0, 0, 0);
            else if (j >= 0) { emit(A_P0, j, 0, 0, b1, 0); emit(A_P1, j, 0, 0, b1, b1); }
            else if (k >= 0) { emit(A_P0, k, 0, 0, b0, 0); emit(A_P1, k, 0, 0, b0, b0); }
            else { emit(A_ZERO, 0, 0, 0, b0 | b1, b0); emit(A_ZERO, 0, 0, 0, b0 | b1, b1); }
            break;
          default: break;
        }
      };
      if (!opt.fused)
        for (int gi : inner) lower(gi);
      for (int gi : post) lower(gi);
      if (pack) {
        // the packed kernel applies the square roots as unscaled rotations; their
        // factors 2^{-1/2} are applied in pairs as exact 1/2 in bulk (a P_SCALE after
        // every kMaxDeferred halves, the remainder at the stage's end), an odd one is
        // carried on, and their phases go to the plan's end (P_GLOBAL); non-diagonal
        // gates, T and two-qubit ops of a packed plan are unconditional
        std::vector<DevOp> ops(P.ops.begin() + ds.op_begin, P.ops.end());
        P.ops.resize(ds.op_begin);
        // condition word: group index bit i <-> tile bit nonr[i], then one bit per
        // non-tile qubit (the tile index)
        int wpos[64];
        for (int q = 0; q < 64; ++q) wpos[q] = -1;
        for (int i = 0; i < group_bits; ++i) wpos[dp.tq[ds.nonr[i]]] = i;
        for (int i = 0; i < dp.nt; ++i) wpos[dp.ntq[i]] = group_bits + i;
        int units = sqrt_carry;  // factors 2^{-1/2} pending
        for (DevOp o : ops) {
          const bool cond_ok = o.cmask == 0 || o.act == A_Z || o.act == A_P0 || o.act == A_P1 ||
                               o.act == A_PHASE || o.act == A_ZERO;
          if (!cond_ok) { *err = "packed plan: conditional op of an unconditional kind"; return false; }
          for (int q = 0; q < n; ++q) {
            if (!((o.cmask >> q) & 1ull)) continue;
            if (wpos[q] < 0 || wpos[q] > 31) { *err = "packed plan: condition outside the condition word"; return false; }
            o.wmask |= 1u << wpos[q];
            if ((o.cval >> q) & 1ull) o.wval |= 1u << wpos[q];
          }
          P.ops.push_back(o);
          if (o.act == A_SX || o.act == A_SY || o.act == A_SXDG || o.act == A_SYDG) {
            phase8 = (phase8 + ((o.act == A_SX || o.act == A_SY) ? 1 : 7)) & 7;
            if (++units == 2 * kMaxDeferred) {
              DevOp sc;
              std::memset(&sc, 0, sizeof(sc));
              sc.act = A_COUNT;
              sc.code = P_SCALE;
              sc.arg = (uint8_t)kMaxDeferred;
              P.ops.push_back(sc);
              units = 0;
            }
          }
        }
        ds.halves = (uint8_t)(units / 2);
        sqrt_carry = units % 2;
      }
      if (P.ops.size() - ds.op_begin > 65535) { *err = "stage too large"; return false; }
      ds.op_count = (uint16_t)(P.ops.size() - ds.op_begin);
      P.stages.push_back(ds);
      P.stage_gates.push_back(inner);
      P.stage_post.push_back(post);
      const int pass_index = (int)P.passes.size();
      for (int gi : inner) { P.order.push_back(gi); P.pass_of.push_back(pass_index); }
      for (int gi : post) { P.order.push_back(gi); P.pass_of.push_back(pass_index); }
    }
    dp.stage_count = (uint16_t)(P.stages.size() - dp.stage_begin);
    {
      bool unitary = true;
      for (int gi : now) {
        const int k = gates[gi].kind;
        if (k == K_P0 || k == K_P1 || k == K_PEQ) unitary = false;
      }
      if (unitary) dp.flags |= PF_UNITARY;
    }
    P.passes.push_back(dp);
    rem.swap(later);
    first_pass = false;
    if (P.passes.size() > 100000) { *err = "planner did not converge"; return false; }
  }
  // the square roots' remaining scalar, e^{i pi phase8/4} 2^{-sqrt_carry/2}, at the end of
  // the last stage (whose ops are the last ones so far)
  if (pack && (phase8 != 0 || sqrt_carry != 0)) {
    if (P.stages.empty() || P.stages.back().op_begin + P.stages.back().op_count != P.ops.size()) {
      *err = "packed plan: no last stage for the square roots' scalar";
      return false;
    }
    DevOp g;
    std::memset(&g, 0, sizeof(g));
    g.act = A_COUNT;
    g.code = P_GLOBAL;
    g.arg = (uint8_t)(phase8 | (sqrt_carry << 3));
    P.ops.push_back(g);
    if (P.stages.back().op_count == 65535) { *err = "stage too large"; return false; }
    P.stages.back().op_count += 1;
  }
  // packed plans: the rounding constant of every T / T-adjoint op (arg 1: the fp32 value
  // above 1/sqrt2, 0: the one below), in plan order, each chosen to bring the running sum
  // of the relative errors back toward zero (see DT1 in tile_pack.cuh)
  if (pack) {
    const double s2 = 0.70710678118654752440;
    const double e_dn = (double)0.70710677f / s2 - 1.0, e_up = (double)0.70710683f / s2 - 1.0;
    double bias = 0.0;
    for (DevOp &o : P.ops) {
      if (o.code < P_DIAG || o.code >= P_DIAG + 12) continue;
      o.arg = bias < 0.0 ? 1 : 0;
      bias += o.arg ? e_up : e_dn;
    }
  }
  // a no-op past the last op: kernels may load the op after a stage's last one
  DevOp end;
  std::memset(&end, 0, sizeof(end));
  end.code = 255;
  end.act = A_COUNT;
  P.ops.push_back(end);
  return true;
}

void stage_unitary(const Plan &P, const std::vector<Gate> &gates, int stage, int r,
                   std::vector<double> *u) {
  const DevStage &ds = P.stages[stage];
  const DevPass *pass = nullptr;
  for (const DevPass &p : P.passes)
    if (stage >= (int)p.stage_begin && stage < (int)(p.stage_begin + p.stage_count)) pass = &p;
  const int d = 1 << r;
  u->assign((size_t)2 * d * d, 0.0);
  for (int i = 0; i < d; ++i) (*u)[2 * ((size_t)i * d + i)] = 1.0;
  int local_of[64];
  for (int q = 0; q < 64; ++q) local_of[q] = -1;
  for (int i = 0; pass && i < pass->m; ++i) local_of[pass->tq[i]] = i;
  // packed plans: matrix bit 0 is tile bit 0 (the pack bit), bit j + 1 register slot j
  const bool packed = pass && (pass->flags & PF_PACKED);
  auto reg_of = [&](int q) {
    if (local_of[q] < 0) return -1;
    if (packed && local_of[q] == 0) return 0;
    for (int j = 0; j < (packed ? r - 1 : r); ++j)
      if (ds.rbit[j] == local_of[q]) return packed ? j + 1 : j;
    return -1;
  };
  for (int gi : P.stage_gates[stage]) {
    const Gate &x = gates[gi];
    if (kind_two_qubit(x.kind)) {
      const int j = reg_of(x.q0), k = reg_of(x.q1);
      for (int row = 0; row < d; ++row) {
        const bool bj = (row >> j) & 1, bk = (row >> k) & 1;
        double s = 1.0;
        if (x.kind == K_CZ && bj && bk) s = -1.0;
        if (x.kind == K_PEQ && bj != bk) s = 0.0;
        for (int col = 0; col < d; ++col) {
          (*u)[2 * ((size_t)row * d + col)] *= s;
          (*u)[2 * ((size_t)row * d + col) + 1] *= s;
        }
      }
      continue;
    }
    double mm[8];
    kind_matrix(x.kind, mm);
    const int j = reg_of(x.q0);
    for (int col = 0; col < d; ++col) {
      for (int row = 0; row < d; ++row) {
        if ((row >> j) & 1) continue;
        const int r1 = row | (1 << j);
        const double xr = (*u)[2 * ((size_t)row * d + col)], xi = (*u)[2 * ((size_t)row * d + col) + 1];
        const double yr = (*u)[2 * ((size_t)r1 * d + col)], yi = (*u)[2 * ((size_t)r1 * d + col) + 1];
        (*u)[2 * ((size_t)row * d + col)] = mm[0] * xr - mm[1] * xi + mm[2] * yr - mm[3] * yi;
        (*u)[2 * ((size_t)row * d + col) + 1] = mm[0] * xi + mm[1] * xr + mm[2] * yi + mm[3] * yr;
        (*u)[2 * ((size_t)r1 * d + col)] = mm[4] * xr - mm[5] * xi + mm[6] * yr - mm[7] * yi;
        (*u)[2 * ((size_t)r1 * d + col) + 1] = mm[4] * xi + mm[5] * xr + mm[6] * yi + mm[7] * yr;
      }
    }
  }
}

}  // namespace svp
