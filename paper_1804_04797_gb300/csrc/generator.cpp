// Seeded random lattice circuit (the gate set and layout of §2: H, T, X^{1/2}, Y^{1/2}
// and CZ between lattice neighbours, CZ positions fixed per layer, layer 0 = H on every
// qubit and not counted in the depth, §1 footnote).  The paper prints neither the CZ
// patterns nor the single-qubit rule; the rules implemented are stated in sv.h.
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/sv.h"
#include "capi_util.h"

namespace {

struct Rng {  // SplitMix64 (Steele, Lea, Flood 2014)
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

struct Bond {
  int a, b;
};

}  // namespace

extern "C" sv_status sv_generate_circuit(const sv_lattice *lat, sv_gate *out, size_t cap,
                                         size_t *n_out) {
  svc::clear_error();
  if (!lat || !n_out) return svc::fail(SV_ERR_ARG, "sv_generate_circuit: null argument");
  const int R = lat->rows, C = lat->cols;
  if (R < 1 || C < 1 || R * C > 64 || lat->depth < 0)
    return svc::fail(SV_ERR_ARG, "sv_generate_circuit: lattice must have 1..64 sites, depth >= 0");
  // qubit number of each site (-1 = removed), row-major over kept sites
  std::vector<int> site(R * C, -1);
  int n = 0;
  for (int i = 0; i < R * C; ++i)
    if (!((lat->removed_mask >> i) & 1ull)) site[i] = n++;
  if (n < 1) return svc::fail(SV_ERR_ARG, "sv_generate_circuit: no qubits left");

  // pattern p in [H0,V0,H1,V1,H2,V2,H3,V3] -> bonds (smaller qubit first)
  std::vector<Bond> pattern[8];
  for (int r = 0; r < R; ++r) {
    for (int c = 0; c < C; ++c) {
      const int a = site[r * C + c];
      if (a < 0) continue;
      if (c + 1 < C && site[r * C + c + 1] >= 0) {
        const int cls = (c + 2 * (r & 1)) & 3;
        pattern[2 * cls].push_back({a, site[r * C + c + 1]});
      }
      if (r + 1 < R && site[(r + 1) * C + c] >= 0) {
        const int cls = (r + 2 * (c & 1)) & 3;
        pattern[2 * cls + 1].push_back({a, site[(r + 1) * C + c]});
      }
    }
  }
  for (auto &p : pattern) {
    for (auto &b : p)
      if (b.a > b.b) { int t = b.a; b.a = b.b; b.b = t; }
    // sort by (a, b): insertion sort, patterns are short
    for (size_t i = 1; i < p.size(); ++i) {
      Bond key = p[i];
      size_t j = i;
      while (j > 0 && (p[j - 1].a > key.a || (p[j - 1].a == key.a && p[j - 1].b > key.b))) {
        p[j] = p[j - 1];
        --j;
      }
      p[j] = key;
    }
  }

  std::vector<sv_gate> g;
  g.reserve((size_t)n * (lat->depth + 1));
  for (int q = 0; q < n; ++q) g.push_back(sv_gate{SV_H, (uint8_t)q, 0, 0, 0});
  Rng rng{lat->seed};
  std::vector<int> last(n, -1);       // previous one-qubit gate kind
  std::vector<char> was_cz(n, 0), is_cz(n, 0);
  static const int kChoices[3] = {SV_T, SV_SX, SV_SY};
  for (int layer = 1; layer <= lat->depth; ++layer) {
    const std::vector<Bond> &pat = pattern[(layer - 1) & 7];
    std::fill(is_cz.begin(), is_cz.end(), 0);
    for (const Bond &b : pat) { is_cz[b.a] = 1; is_cz[b.b] = 1; }
    for (int q = 0; q < n; ++q) {
      if (!was_cz[q] || is_cz[q]) continue;
      int cand[3], nc = 0;
      for (int k : kChoices)
        if (k != last[q]) cand[nc++] = k;
      const uint64_t draw = rng.next();
      const int kind = cand[draw % (uint64_t)nc];
      last[q] = kind;
      g.push_back(sv_gate{(uint8_t)kind, (uint8_t)q, 0, 0, (uint32_t)layer});
    }
    for (const Bond &b : pat)
      g.push_back(sv_gate{SV_CZ, (uint8_t)b.a, (uint8_t)b.b, 0, (uint32_t)layer});
    was_cz.swap(is_cz);
  }
  *n_out = g.size();
  if (out) {
    if (cap < g.size()) return svc::fail(SV_ERR_ARG, "sv_generate_circuit: cap too small");
    std::memcpy(out, g.data(), g.size() * sizeof(sv_gate));
  }
  return SV_OK;
}
