// build_regular.cpp -- ldpc_code_build_regular: a seeded random (dv, dc)-regular
// Tanner graph (the regular (3,6) code of the paper's small experiments is of
// this kind; Sec. 2.A defines the graph, Sec. 5 the workloads).
//
// Construction: dv sockets per variable node and dc per check node; the check
// sockets are shuffled (Fisher-Yates) and matched in order to the variable
// sockets.  Double edges, and with `girth6` the 4-cycles, are then removed by
// seeded swaps of the check endpoints of two edges: one edge is drawn among
// those that take part in a double edge or a 4-cycle, the other among all
// edges, and the swap is kept when it does not raise the count of double
// edges plus 4-cycles (degrees never change).  Random numbers come from
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), written from its published
// definition, seeded with `seed`; integers below r by rejection of the biased
// top range.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "ldpc.h"

namespace {

struct SplitMix64 {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint64_t below(uint64_t r) {  // uniform in [0, r), r > 0
    const uint64_t lim = UINT64_MAX - UINT64_MAX % r;
    uint64_t v;
    do v = next();
    while (v >= lim);
    return v % r;
  }
};

// Count of double edges plus (if cycles) 4-cycles of the graph cn[e] -- vn[e],
// and the mark of every edge that takes part in one.
struct Cost {
  int32_t m, n;
  bool cycles;
  std::vector<std::vector<int32_t>> cn_vars;  // variables of each check (with repeats)
  std::vector<std::vector<int32_t>> vn_checks;
  std::vector<int32_t> overlap;
  std::vector<int32_t> touched;

  int64_t eval(const std::vector<int32_t>& cn, const std::vector<int32_t>& vn, std::vector<uint8_t>* bad) {
    for (auto& v : cn_vars) v.clear();
    for (auto& v : vn_checks) v.clear();
    for (size_t e = 0; e < cn.size(); ++e) {
      cn_vars[cn[e]].push_back(vn[e]);
      vn_checks[vn[e]].push_back(cn[e]);
    }
    int64_t cost = 0;
    if (bad) bad->assign(cn.size(), 0);
    // double edges: a variable listed twice in a check
    std::vector<int32_t> seen((size_t)n, -1);
    for (int32_t c = 0; c < m; ++c)
      for (int32_t v : cn_vars[c]) {
        if (seen[v] == c) ++cost;
        seen[v] = c;
      }
    std::vector<uint8_t> dbl_c((size_t)m, 0);
    std::fill(seen.begin(), seen.end(), -1);
    for (int32_t c = 0; c < m; ++c)
      for (int32_t v : cn_vars[c]) {
        if (seen[v] == c) dbl_c[c] = 1;
        seen[v] = c;
      }
    // 4-cycles: check pairs (c1 < c2) sharing s >= 2 distinct variables give s(s-1)/2
    std::vector<uint8_t> in4((size_t)m, 0);
    if (cycles) {
      for (int32_t c1 = 0; c1 < m; ++c1) {
        touched.clear();
        std::vector<int32_t> vs = cn_vars[c1];
        std::sort(vs.begin(), vs.end());
        vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
        for (int32_t v : vs) {
          std::vector<int32_t> cs = vn_checks[v];
          std::sort(cs.begin(), cs.end());
          cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
          for (int32_t c2 : cs) {
            if (c2 <= c1) continue;
            if (overlap[c2]++ == 0) touched.push_back(c2);
          }
        }
        for (int32_t c2 : touched) {
          const int64_t s = overlap[c2];
          if (s >= 2) {
            cost += s * (s - 1) / 2;
            in4[c1] = 1;
            in4[c2] = 1;
          }
          overlap[c2] = 0;
        }
      }
    }
    if (bad) {
      // an edge is bad when its check has a double edge, or its check is in a
      // 4-cycle with another check through this edge's variable
      for (size_t e = 0; e < cn.size(); ++e) {
        const int32_t c = cn[e], v = vn[e];
        bool b = dbl_c[c] != 0;
        if (!b && cycles && in4[c]) {
          for (int32_t c2 : vn_checks[v]) {
            if (c2 == c || !in4[c2]) continue;
            // c and c2 share v; bad if they share another variable too
            int shared = 0;
            for (int32_t w : cn_vars[c2])
              if (w != v && std::find(cn_vars[c].begin(), cn_vars[c].end(), w) != cn_vars[c].end()) {
                shared = 1;
                break;
              }
            if (shared) {
              b = true;
              break;
            }
          }
        }
        (*bad)[e] = b;
      }
    }
    return cost;
  }
};

}  // namespace

extern "C" ldpc_status_t ldpc_code_build_regular(int32_t n, int32_t dv, int32_t dc, uint64_t seed, int32_t girth6,
                                                 int32_t k_info, ldpc_code_t** out) {
  if (!out) {
    ldpc::set_error_detail("out is NULL");
    return LDPC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (n <= 0 || dv <= 0 || dc <= 1 || dv > 32 || dc > 32 || ((int64_t)n * dv) % dc != 0 || n > (1 << 22)) {
    ldpc::set_error_detail("need n > 0, 0 < dv <= 32, 1 < dc <= 32, n dv a multiple of dc, n <= 2^22");
    return LDPC_ERR_INVALID_ARG;
  }
  const int32_t m = (int32_t)((int64_t)n * dv / dc);
  if (dc > n || dv > m) {
    ldpc::set_error_detail("degrees larger than the other side");
    return LDPC_ERR_INVALID_ARG;
  }
  const int64_t E = (int64_t)n * dv;
  std::vector<int32_t> vn((size_t)E), cn((size_t)E);
  for (int64_t e = 0; e < E; ++e) {
    vn[(size_t)e] = (int32_t)(e / dv);
    cn[(size_t)e] = (int32_t)(e / dc);
  }
  SplitMix64 rng{seed};
  for (int64_t i = E - 1; i > 0; --i) std::swap(cn[(size_t)i], cn[(size_t)rng.below((uint64_t)i + 1)]);
  Cost cc;
  cc.m = m;
  cc.n = n;
  cc.cycles = girth6 != 0;
  cc.cn_vars.resize((size_t)m);
  cc.vn_checks.resize((size_t)n);
  cc.overlap.assign((size_t)m, 0);
  std::vector<uint8_t> bad, bad2;
  int64_t cost = cc.eval(cn, vn, &bad);
  const int64_t max_iter = 200000;
  for (int64_t it = 0; cost > 0 && it < max_iter; ++it) {
    std::vector<int64_t> cand;
    for (int64_t e = 0; e < E; ++e)
      if (bad[(size_t)e]) cand.push_back(e);
    if (cand.empty()) break;
    const int64_t a = cand[(size_t)rng.below((uint64_t)cand.size())];
    const int64_t b = (int64_t)rng.below((uint64_t)E);
    if (cn[(size_t)a] == cn[(size_t)b]) continue;
    std::swap(cn[(size_t)a], cn[(size_t)b]);
    const int64_t c2 = cc.eval(cn, vn, &bad2);
    if (c2 <= cost) {
      cost = c2;
      bad.swap(bad2);
    } else {
      std::swap(cn[(size_t)a], cn[(size_t)b]);
    }
  }
  if (cost > 0) {
    ldpc::set_error_detail("could not remove double edges / 4-cycles (" + std::to_string(cost) + " left)");
    return LDPC_ERR_UNSUPPORTED;
  }
  return ldpc_code_create(cn.data(), vn.data(), E, m, n, nullptr, k_info > 0 ? k_info : n - m, out);
}
