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

// Explicit entries of a slab by their three edge materials: open addressing
// with linear probing over entry numbers (slot = number + 1, 0 = empty), the
// keys kept in insertion order, so an entry's number is its insertion rank.
// The key bits are mixed with the splitmix64 finalizer (Steele, Lea and
// Flood, OOPSLA 2014): doubles from float data end in many zero bits, which a
// power-of-two table would otherwise see as one cluster.
class TripleIndex {
 public:
  // Number of `k`, inserting it as the next number if new (`inserted`).
  uint32_t find_or_insert(const TripleKey& k, bool& inserted) {
    if (2 * (keys_.size() + 1) > slot_.size()) grow();
    size_t h = hash(k) & mask_;
    for (;;) {
      const uint32_t v = slot_[h];
      if (v == 0) {
        keys_.push_back(k);
        slot_[h] = (uint32_t)keys_.size();
        inserted = true;
        return (uint32_t)keys_.size() - 1;
      }
      if (keys_[v - 1] == k) {
        inserted = false;
        return v - 1;
      }
      h = (h + 1) & mask_;
    }
  }

 private:
  void grow() {
    const size_t n = slot_.empty() ? 1024 : 2 * slot_.size();
    slot_.assign(n, 0);
    mask_ = n - 1;
    for (size_t q = 0; q < keys_.size(); ++q) {
      size_t h = hash(keys_[q]) & mask_;
      while (slot_[h] != 0) h = (h + 1) & mask_;
      slot_[h] = (uint32_t)q + 1;
    }
  }
  static uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  static size_t hash(const TripleKey& k) {
    uint64_t h = 0;
    for (int c = 0; c < 3; ++c) h = mix(mix(h ^ k.k[c].e) ^ k.k[c].s);
    return (size_t)h;
  }
  std::vector<TripleKey> keys_;
  std::vector<uint32_t> slot_;
  size_t mask_ = 0;
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

// Per-cell materials of one grid (x fastest; null eps = vacuum, null sigma =
// lossless). The material of an interior edge is the mean (eps, sigma) of its
// four cells, summed in double in the fixed order (-,-), (+,-), (-,+), (+,+)
// of the two transverse offsets (edge_row_means). A cell with eps = +inf
// (perfect conductor) makes the mean infinite: PEC edge.
struct EdgeMaterials {
  const Dims& d;
  const float* eps;
  const float* sig;
};

using FreqMap = std::unordered_map<EdgeKey, long long, EdgeKeyHash>;
using ClassMap = std::unordered_map<EdgeKey, int, EdgeKeyHash>;

// Valid i range [i0, i1) of component c's interior edges on row (j, k);
// empty when the row has none.
void edge_row_range(const Dims& d, int c, int j, int k, int& i0, int& i1) {
  const bool ok = c == 0 ? (j >= 1 && j < d.ny && k >= 1 && k < d.nz)
                  : c == 1 ? (j < d.ny && k >= 1 && k < d.nz)
                           : (j >= 1 && j < d.ny && k < d.nz);
  i0 = c == 0 ? 0 : 1;
  i1 = ok ? d.nx : i0;
}

// Edge means of component c along row (j, k) for i in [i0, i1), written to
// e[i], s[i]: each the four-cell sum in the order above, times 1/4. The four cell rows are the (-,-), (+,-), (-,+), (+,+) offsets of
// the two transverse axes; along x an offset is a shift of the row pointer.
void edge_row_means(const EdgeMaterials& m, int c, int j, int k, int i0, int i1, double* e, double* s) {
  const Dims& d = m.d;
  // cell rows (j', k') and x shifts of the four terms, in summation order
  int jr[4], kr[4], sh[4];
  if (c == 0) {  // (i, j-1, k-1), (i, j, k-1), (i, j-1, k), (i, j, k)
    const int J[4] = {j - 1, j, j - 1, j}, K[4] = {k - 1, k - 1, k, k}, X[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) { jr[q] = J[q]; kr[q] = K[q]; sh[q] = X[q]; }
  } else if (c == 1) {  // (i-1, j, k-1), (i, j, k-1), (i-1, j, k), (i, j, k)
    const int J[4] = {j, j, j, j}, K[4] = {k - 1, k - 1, k, k}, X[4] = {-1, 0, -1, 0};
    for (int q = 0; q < 4; ++q) { jr[q] = J[q]; kr[q] = K[q]; sh[q] = X[q]; }
  } else {  // (i-1, j-1, k), (i, j-1, k), (i-1, j, k), (i, j, k)
    const int J[4] = {j - 1, j - 1, j, j}, K[4] = {k, k, k, k}, X[4] = {-1, 0, -1, 0};
    for (int q = 0; q < 4; ++q) { jr[q] = J[q]; kr[q] = K[q]; sh[q] = X[q]; }
  }
  auto rowp = [&](const float* a, int q) { return a + ((long long)kr[q] * d.ny + jr[q]) * d.nx + sh[q]; };
  if (m.eps) {
    const float *a0 = rowp(m.eps, 0), *a1 = rowp(m.eps, 1), *a2 = rowp(m.eps, 2), *a3 = rowp(m.eps, 3);
    for (int i = i0; i < i1; ++i)
      e[i] = ((((double)a0[i] + (double)a1[i]) + (double)a2[i]) + (double)a3[i]) * 0.25;
  } else {
    for (int i = i0; i < i1; ++i) e[i] = (((1.0 + 1.0) + 1.0) + 1.0) * 0.25;
  }
  if (m.sig) {
    const float *b0 = rowp(m.sig, 0), *b1 = rowp(m.sig, 1), *b2 = rowp(m.sig, 2), *b3 = rowp(m.sig, 3);
    for (int i = i0; i < i1; ++i)
      s[i] = ((((double)b0[i] + (double)b1[i]) + (double)b2[i]) + (double)b3[i]) * 0.25;
  } else {
    for (int i = i0; i < i1; ++i) s[i] = (((0.0 + 0.0) + 0.0) + 0.0) * 0.25;
  }
}

// Frequency of every edge material on planes [k0, k1) (runs along x at once).
void count_slab(const EdgeMaterials& m, int k0, int k1, FreqMap& freq) {
  const Dims& d = m.d;
  std::vector<double> e(d.nx + 1), s(d.nx + 1);
  for (int c = 0; c < 3; ++c) {
    EdgeKey last{~0ull, ~0ull};
    long long run = 0;
    for (int k = k0; k < k1; ++k)
      for (int j = 0; j <= d.ny; ++j) {
        int i0, i1;
        edge_row_range(d, c, j, k, i0, i1);
        if (i0 >= i1) continue;
        edge_row_means(m, c, j, k, i0, i1, e.data(), s.data());
        for (int i = i0; i < i1; ++i) {
          if (std::isinf(e[i])) continue;
          const EdgeKey key{dbits(e[i]), dbits(s[i])};
          if (key == last) {
            ++run;
            continue;
          }
          if (run) freq[last] += run;
          last = key;
          run = 1;
        }
      }
    if (run) freq[last] += run;
  }
}

// Words of planes [k0, k1); explicit entries go to `t` (indices local to the
// slab). Returns false if the slab needs more than 2^29 entries.
bool words_slab(const EdgeMaterials& m, double dt, double S64, const ClassMap& cls, int k0, int k1,
                uint32_t* words, MaterialTables& t) {
  const Dims& d = m.d;
  TripleIndex expl;
  EdgeKey lk[3] = {{~0ull, ~0ull}, {~0ull, ~0ull}, {~0ull, ~0ull}};
  int lc[3] = {-1, -1, -1};
  std::vector<double> eb[3], sb[3];
  for (int c = 0; c < 3; ++c) {
    eb[c].resize(d.nx + 1);
    sb[c].resize(d.nx + 1);
  }
  for (int k = k0; k < k1; ++k)
    for (int j = 0; j <= d.ny; ++j) {
      uint32_t* row = words + ((long long)k * d.ny1 + j) * d.nxp;
      int r0[3], r1[3];
      for (int c = 0; c < 3; ++c) {
        edge_row_range(d, c, j, k, r0[c], r1[c]);
        if (r0[c] < r1[c]) edge_row_means(m, c, j, k, r0[c], r1[c], eb[c].data(), sb[c].data());
      }
      for (int i = 0; i < d.nxp; ++i) {
        int ci[3] = {0, 0, 0};
        TripleKey tk{{{0, 0}, {0, 0}, {0, 0}}};
        bool explicit_pt = false;
        for (int c = 0; c < 3; ++c) {
          if (i < r0[c] || i >= r1[c]) continue;
          const double e = eb[c][i], s = sb[c][i];
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
        bool inserted = false;
        const uint32_t q = expl.find_or_insert(tk, inserted);
        if (q >= (1u << 29)) return false;
        if (inserted) {
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

long long first_bad_material(const float* eps, const float* sig, long long n, int nthreads) {
  nthreads = std::max(1, nthreads);
  std::vector<long long> bad(nthreads, -1);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      const long long c0 = n * t / nthreads, c1 = n * (t + 1) / nthreads;
      for (long long c = c0; c < c1; ++c)
        if ((eps && !(eps[c] >= 1.0f)) || (sig && (!(sig[c] >= 0.0f) || !std::isfinite(sig[c])))) {
          bad[t] = c;
          break;
        }
    });
  for (std::thread& x : th) x.join();
  for (long long c : bad)
    if (c >= 0) return c;
  return -1;
}

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
