// Host construction of the per-point material words and coefficient tables
// (the edge materials of the Sec. 2.1 scheme), shared by single grids and
// batches of cavities.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sophie_internal.h"

namespace sophie {

namespace {

constexpr double kEps0 = 8.8541878128e-12;

struct EdgeKey {
  uint64_t e, s;
  bool operator==(const EdgeKey& o) const { return e == o.e && s == o.s; }
};
struct EdgeKeyHash {
  size_t operator()(const EdgeKey& k) const {
    return (size_t)(k.e * 0x9E3779B97F4A7C15ull ^ (k.s + 0x632BE59BD9B4E019ull + (k.e << 6)));
  }
};

// The three edge materials of one explicit point.
struct TripleKey {
  EdgeKey k[3];
  bool operator==(const TripleKey& o) const { return k[0] == o.k[0] && k[1] == o.k[1] && k[2] == o.k[2]; }
};
struct TripleKeyHash {
  size_t operator()(const TripleKey& t) const {
    EdgeKeyHash h;
    return h(t.k[0]) * 31u + h(t.k[1]) * 17u + h(t.k[2]);
  }
};

uint64_t dbits(double v) {
  uint64_t u;
  memcpy(&u, &v, 8);
  return u;
}

double from_bits(uint64_t u) {
  double v;
  memcpy(&v, &u, 8);
  return v;
}

bool edge_interior(const Dims& d, int c, int i, int j, int k) {
  switch (c) {
    case 0: return i >= 0 && i < d.nx && j >= 1 && j < d.ny && k >= 1 && k < d.nz;
    case 1: return i >= 1 && i < d.nx && j >= 0 && j < d.ny && k >= 1 && k < d.nz;
    default: return i >= 1 && i < d.nx && j >= 1 && j < d.ny && k >= 0 && k < d.nz;
  }
}

}  // namespace

double source_waveform(int kind, double amp, double f0, double bw, double t0, double dt, long long n) {
  const double pi = 3.14159265358979323846;
  const double sf = bw / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  const double st = 1.0 / (2.0 * pi * sf);
  const double t = ((double)n + 0.5) * dt;
  const double u = t - t0;
  const double env = std::exp(-(u * u) / (2.0 * st * st));
  return amp * (kind == 0 ? std::sin(2.0 * pi * f0 * u) * env : env);
}

float2 edge_coefficients(double dt, double S64, double e, double s) {
  const double beta = (s * dt) / (2.0 * kEps0 * e);
  const double ca = (1.0 - beta) / (1.0 + beta);
  const double cb = (S64 / e) / (1.0 + beta);
  return make_float2((float)ca, (float)cb);
}

namespace {

// Edge materials of one grid: mean (eps, sigma) of an interior edge, four
// cells summed in the fixed order (-,-), (+,-), (-,+), (+,+) of the two
// transverse offsets. A cell with eps = +inf (perfect conductor) makes the
// mean infinite: PEC edge.
struct EdgeMaterials {
  const Dims& d;
  const float* eps;
  const float* sig;
  double E(int i, int j, int k) const { return eps ? (double)eps[((long long)k * d.ny + j) * d.nx + i] : 1.0; }
  double Sg(int i, int j, int k) const { return sig ? (double)sig[((long long)k * d.ny + j) * d.nx + i] : 0.0; }
  void mean(int c, int i, int j, int k, double& e, double& s) const {
    double e4, s4;
    if (c == 0) {
      e4 = ((E(i, j - 1, k - 1) + E(i, j, k - 1)) + E(i, j - 1, k)) + E(i, j, k);
      s4 = ((Sg(i, j - 1, k - 1) + Sg(i, j, k - 1)) + Sg(i, j - 1, k)) + Sg(i, j, k);
    } else if (c == 1) {
      e4 = ((E(i - 1, j, k - 1) + E(i, j, k - 1)) + E(i - 1, j, k)) + E(i, j, k);
      s4 = ((Sg(i - 1, j, k - 1) + Sg(i, j, k - 1)) + Sg(i - 1, j, k)) + Sg(i, j, k);
    } else {
      e4 = ((E(i - 1, j - 1, k) + E(i, j - 1, k)) + E(i - 1, j, k)) + E(i, j, k);
      s4 = ((Sg(i - 1, j - 1, k) + Sg(i, j - 1, k)) + Sg(i - 1, j, k)) + Sg(i, j, k);
    }
    e = e4 * 0.25;
    s = s4 * 0.25;
  }
};

using FreqMap = std::unordered_map<EdgeKey, long long, EdgeKeyHash>;
using ClassMap = std::unordered_map<EdgeKey, int, EdgeKeyHash>;

// Frequency of every edge material on planes [k0, k1) (runs along x at once).
void count_slab(const EdgeMaterials& m, int k0, int k1, FreqMap& freq) {
  const Dims& d = m.d;
  for (int c = 0; c < 3; ++c) {
    EdgeKey last{~0ull, ~0ull};
    long long run = 0;
    for (int k = k0; k < k1; ++k)
      for (int j = 0; j <= d.ny; ++j)
        for (int i = 0; i <= d.nx; ++i) {
          if (!edge_interior(d, c, i, j, k)) continue;
          double e, s;
          m.mean(c, i, j, k, e, s);
          if (std::isinf(e)) continue;
          const EdgeKey key{dbits(e), dbits(s)};
          if (key == last) {
            ++run;
            continue;
          }
          if (run) freq[last] += run;
          last = key;
          run = 1;
        }
    if (run) freq[last] += run;
  }
}

// Words of planes [k0, k1); explicit entries go to `t` (indices local to the
// slab). Returns false if the slab needs more than 2^29 entries.
bool words_slab(const EdgeMaterials& m, double dt, double S64, const ClassMap& cls, int k0, int k1,
                uint32_t* words, MaterialTables& t) {
  const Dims& d = m.d;
  std::unordered_map<TripleKey, uint32_t, TripleKeyHash> expl;
  EdgeKey lk[3] = {{~0ull, ~0ull}, {~0ull, ~0ull}, {~0ull, ~0ull}};
  int lc[3] = {-1, -1, -1};
  for (int k = k0; k < k1; ++k)
    for (int j = 0; j <= d.ny; ++j) {
      uint32_t* row = words + ((long long)k * d.ny1 + j) * d.nxp;
      for (int i = 0; i < d.nxp; ++i) {
        int ci[3] = {0, 0, 0};
        TripleKey tk{{{0, 0}, {0, 0}, {0, 0}}};
        bool explicit_pt = false;
        for (int c = 0; c < 3; ++c) {
          if (!edge_interior(d, c, i, j, k)) continue;
          double e, s;
          m.mean(c, i, j, k, e, s);
          if (std::isinf(e)) continue;  // PEC: class 0
          const EdgeKey key{dbits(e), dbits(s)};
          tk.k[c] = key;
          if (!(key == lk[c])) {
            auto it = cls.find(key);
            lk[c] = key;
            lc[c] = it == cls.end() ? -1 : it->second;
          }
          ci[c] = lc[c];
          if (ci[c] < 0) explicit_pt = true;
        }
        if (!explicit_pt) {
          row[i] = cls_word((uint32_t)ci[0], (uint32_t)ci[1], (uint32_t)ci[2]);
          continue;
        }
        auto it = expl.find(tk);
        uint32_t q;
        if (it != expl.end()) {
          q = it->second;
        } else {
          q = (uint32_t)(t.eeps.size() / 3);
          if (q >= (1u << 29)) return false;
          expl.emplace(tk, q);
          for (int c = 0; c < 3; ++c) {
            const bool in = tk.k[c].e != 0 || tk.k[c].s != 0;
            const double e = from_bits(tk.k[c].e), s = from_bits(tk.k[c].s);
            t.ecoef.push_back(in ? edge_coefficients(dt, S64, e, s) : make_float2(0.f, 0.f));
            t.eeps.push_back(in ? e : 0.0);
            t.esig.push_back(in ? s : 0.0);
          }
        }
        row[i] = kExpFlag | (q << 3);
      }
    }
  return true;
}

// Run f(slab) for slab = 0 .. nslab-1 on up to nthreads threads.
template <class F>
void for_slabs(int nslab, int nthreads, F&& f) {
  if (nthreads <= 1 || nslab <= 1) {
    for (int s = 0; s < nslab; ++s) f(s);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < std::min(nthreads, nslab); ++t)
    th.emplace_back([&]() {
      for (int s = next.fetch_add(1); s < nslab; s = next.fetch_add(1)) f(s);
    });
  for (std::thread& t : th) t.join();
}

}  // namespace

int build_material_tables(const Dims& d, double dt, double S64, const float* eps, const float* sig, uint32_t* words,
                          MaterialTables* out, int nthreads) {
  const EdgeMaterials m{d, eps, sig};
  // Slabs of z planes fixed by the grid alone (the tables do not depend on the
  // thread count): at most 64, each at least 16 planes thick, so that the
  // points of a slab that share three edge materials (e.g. the planes of one
  // material block) share one explicit entry and its cache lines.
  const int nslab = std::max(1, std::min(64, d.nz1 / 16));
  auto slab_k = [&](int s) { return (int)((long long)d.nz1 * s / nslab); };
  // Pass 1: frequencies per slab, merged.
  std::vector<FreqMap> fs(nslab);
  for_slabs(nslab, nthreads, [&](int s) { count_slab(m, slab_k(s), slab_k(s + 1), fs[s]); });
  FreqMap freq;
  for (const FreqMap& f : fs)
    for (const auto& kv : f) freq[kv.first] += kv.second;
  fs.clear();
  // Classes: the most frequent materials (class 0 is PEC / absent).
  std::vector<std::pair<long long, EdgeKey>> order;
  order.reserve(freq.size());
  for (const auto& kv : freq) order.push_back({kv.second, kv.first});
  std::sort(order.begin(), order.end(), [](const std::pair<long long, EdgeKey>& a, const std::pair<long long, EdgeKey>& b) {
    if (a.first != b.first) return a.first > b.first;
    return a.second.e != b.second.e ? a.second.e < b.second.e : a.second.s < b.second.s;
  });
  MaterialTables t;
  ClassMap cls;
  t.coef.assign(1, make_float2(0.f, 0.f));
  t.eps.assign(1, 0.0);
  t.sig.assign(1, 0.0);
  for (size_t q = 0; q < order.size() && (int)t.coef.size() < kMaxClasses; ++q) {
    const double e = from_bits(order[q].second.e), s = from_bits(order[q].second.s);
    cls.emplace(order[q].second, (int)t.coef.size());
    t.coef.push_back(edge_coefficients(dt, S64, e, s));
    t.eps.push_back(e);
    t.sig.push_back(s);
  }
  // Pass 2: words per slab; a point with an edge outside the classes gets an
  // explicit entry, shared by the slab's points with the same three edge
  // materials. Slab-local indices are then shifted by the slab's offset.
  std::vector<MaterialTables> st(nslab);
  std::atomic<bool> ok(true);
  for_slabs(nslab, nthreads, [&](int s) {
    if (!words_slab(m, dt, S64, cls, slab_k(s), slab_k(s + 1), words, st[s])) ok.store(false);
  });
  if (!ok.load()) return -1;
  std::vector<size_t> off(nslab + 1, 0);
  for (int s = 0; s < nslab; ++s) off[s + 1] = off[s] + st[s].eeps.size() / 3;
  if (off[nslab] >= (1u << 29)) return -1;
  for_slabs(nslab, nthreads, [&](int s) {
    if (!off[s]) return;
    const uint32_t add = (uint32_t)off[s] << 3;
    uint32_t* w = words + (long long)slab_k(s) * d.ny1 * d.nxp;
    const long long n = (long long)(slab_k(s + 1) - slab_k(s)) * d.ny1 * d.nxp;
    for (long long q = 0; q < n; ++q)
      if (w[q] & kExpFlag) w[q] += add;
  });
  t.ecoef.reserve(off[nslab] * 3);
  t.eeps.reserve(off[nslab] * 3);
  t.esig.reserve(off[nslab] * 3);
  for (int s = 0; s < nslab; ++s) {
    t.ecoef.insert(t.ecoef.end(), st[s].ecoef.begin(), st[s].ecoef.end());
    t.eeps.insert(t.eeps.end(), st[s].eeps.begin(), st[s].eeps.end());
    t.esig.insert(t.esig.end(), st[s].esig.begin(), st[s].esig.end());
  }
  *out = std::move(t);
  return 0;
}

}  // namespace sophie
