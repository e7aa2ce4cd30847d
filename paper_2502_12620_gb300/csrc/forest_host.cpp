// Host-side block forest (see forest_host.hpp for the paper references).
#include "forest_host.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>

namespace dgf {

// ------------------------------------------------------------------ basis
double legendre(int k, double x) {
  if (k == 0) return 1.0;
  double a = 1.0, b = x;
  for (int j = 1; j < k; ++j) {
    double c = ((2 * j + 1) * x * b - j * a) / (j + 1);
    a = b;
    b = c;
  }
  return b;
}

double legendre_deriv(int k, double x) {
  // P'_{j+1} = P'_{j-1} + (2j+1) P_j
  if (k == 0) return 0.0;
  double dm1 = 0.0, d0 = 1.0;  // P'_0, P'_1
  for (int j = 1; j < k; ++j) {
    double d1 = dm1 + (2 * j + 1) * legendre(j, x);
    dm1 = d0;
    d0 = d1;
  }
  return d0;
}

static void gauss_rule(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N, 0.0);
  w.assign(N, 0.0);
  for (int i = 0; i < N; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (N + 0.5));
    for (int it = 0; it < 100; ++it) {
      double dz = legendre(N, z) / legendre_deriv(N, z);
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double dp = legendre_deriv(N, z);
    x[N - 1 - i] = z;  // ascending order
    w[N - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void Basis1D::build(int N_) {
  N = N_;
  gauss_rule(N, x, w);
  V.assign(N * N, 0.0);
  Vi.assign(N * N, 0.0);
  for (int q = 0; q < N; ++q)
    for (int k = 0; k < N; ++k) {
      V[q * N + k] = legendre(k, x[q]);
      Vi[k * N + q] = 0.5 * (2 * k + 1) * w[q] * legendre(k, x[q]);
    }
  Dn.assign(N * N, 0.0);
  for (int q = 0; q < N; ++q)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += Vi[k * N + j] * legendre_deriv(k, x[q]);
      Dn[q * N + j] = s;
    }
  Sh.assign(N * N, 0.0);
  for (int q = 0; q < N; ++q)
    for (int j = 0; j < N; ++j) Sh[q * N + j] = (w[j] / w[q]) * Dn[j * N + q];
  lp.assign(N, 0.0);
  lm.assign(N, 0.0);
  for (int q = 0; q < N; ++q) {
    double sp = 0.0, sm = 0.0;
    for (int k = 0; k < N; ++k) {
      sp += Vi[k * N + q];
      sm += Vi[k * N + q] * ((k & 1) ? -1.0 : 1.0);
    }
    lp[q] = sp;
    lm[q] = sm;
  }
  // split matrices by an exact (N+1)-point rule
  std::vector<double> xx, ww;
  gauss_rule(N + 1, xx, ww);
  Sm.assign(N * N, 0.0);
  Sp.assign(N * N, 0.0);
  for (int l = 0; l < N; ++l)
    for (int k = 0; k < N; ++k) {
      double am = 0.0, ap = 0.0;
      for (size_t i = 0; i < xx.size(); ++i) {
        am += ww[i] * legendre(l, xx[i]) * legendre(k, 0.5 * (xx[i] - 1.0));
        ap += ww[i] * legendre(l, xx[i]) * legendre(k, 0.5 * (xx[i] + 1.0));
      }
      Sm[l * N + k] = 0.5 * (2 * l + 1) * am;
      Sp[l * N + k] = 0.5 * (2 * l + 1) * ap;
    }
  Snm.assign(N * N, 0.0);
  Snp.assign(N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      Snm[i * N + j] = lagrange(j, 0.5 * (x[i] - 1.0));
      Snp[i * N + j] = lagrange(j, 0.5 * (x[i] + 1.0));
    }
}

double Basis1D::lagrange(int j, double xi) const {
  double s = 0.0;
  for (int k = 0; k < N; ++k) s += Vi[k * N + j] * legendre(k, xi);
  return s;
}

// -------------------------------------------------------------- orientation
static const int kPerm2[2][2] = {{0, 1}, {1, 0}};
static const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

int orient_code(const Orient& o, int d) {
  int idx = -1;
  int np = d == 2 ? 2 : 6;
  for (int i = 0; i < np && idx < 0; ++i) {
    bool eq = true;
    for (int a = 0; a < d; ++a) eq = eq && ((d == 2 ? kPerm2[i][a] : kPerm3[i][a]) == o.pi[a]);
    if (eq) idx = i;
  }
  int bits = 0;
  for (int a = 0; a < d; ++a)
    if (o.sg[a] < 0) bits |= 1 << a;
  return idx * (1 << d) + bits;
}

Orient orient_from_code(int code, int d) {
  Orient o;
  int idx = code >> d, bits = code & ((1 << d) - 1);
  for (int a = 0; a < d; ++a) {
    o.pi[a] = d == 2 ? kPerm2[idx][a] : kPerm3[idx][a];
    o.sg[a] = ((bits >> a) & 1) ? -1 : 1;
  }
  return o;
}

// ------------------------------------------------------------------- keys
uint64_t Forest::key(int64_t root, int level, const int* pos) {
  return ((uint64_t)root << 38) | ((uint64_t)level << 33) | (uint64_t)pos[0] |
         ((uint64_t)pos[1] << 11) | ((uint64_t)pos[2] << 22);
}

void Forest::unkey(uint64_t k, int64_t* root, int* level, int* pos) {
  *root = (int64_t)(k >> 38);
  *level = (int)((k >> 33) & 31);
  pos[0] = (int)(k & 2047);
  pos[1] = (int)((k >> 11) & 2047);
  pos[2] = (int)((k >> 22) & 2047);
}

// ------------------------------------------------------------------- init
bool Forest::init(int dim, int n_seg, int deg, int64_t n_nodes, const double* xyz, int64_t n_roots,
                  const int64_t* corners, const double* cell_nodes, int n_per, const double* per) {
  if (dim != 2 && dim != 3) return error = "dim must be 2 or 3", false;
  if (n_seg < 2 || n_seg > 16 || (n_seg & 1)) return error = "n_seg must be even in [2,16]", false;
  if (deg < 0 || deg > 3) return error = "p must be in [0,3]", false;
  if (n_roots <= 0 || n_nodes <= 0 || !xyz || !corners) return error = "empty forest", false;
  if (n_per < 0 || n_per > 3) return error = "n_periodic must be 0..3", false;
  d = dim;
  n = n_seg;
  p = deg;
  R = n_roots;
  const int nc = 1 << d;
  nodes.assign(xyz, xyz + n_nodes * d);
  root_corners.assign(corners, corners + n_roots * nc);
  for (int64_t c : root_corners)
    if (c < 0 || c >= n_nodes) return error = "root corner id out of range", false;
  n_periodic = n_per;
  periodic.assign(per, per + n_per * d);
  const int nn = (int)std::pow(n + 1, d);
  root_nodes.assign(R, std::vector<double>(nn * d, 0.0));
  for (int64_t r = 0; r < R; ++r) {
    if (cell_nodes) {
      std::memcpy(root_nodes[r].data(), cell_nodes + r * nn * d, sizeof(double) * nn * d);
      continue;
    }
    for (int li = 0; li < nn; ++li) {
      double xi[3];
      int t = li;
      for (int a = 0; a < d; ++a) {
        xi[a] = -1.0 + 2.0 * (t % (n + 1)) / n;
        t /= (n + 1);
      }
      for (int k = 0; k < nc; ++k) {
        double wgt = 1.0;
        for (int a = 0; a < d; ++a) wgt *= 0.5 * (1.0 + (((k >> a) & 1) ? 1.0 : -1.0) * xi[a]);
        for (int j = 0; j < d; ++j) root_nodes[r][li * d + j] += wgt * nodes[root_corners[r * nc + k] * d + j];
      }
    }
  }
  if (!match_root_faces()) return false;
  tree.clear();
  int z[3] = {0, 0, 0};
  for (int64_t r = 0; r < R; ++r) tree[key(r, 1, z)] = 1;
  order_leaves();
  return true;
}

bool Forest::match_root_faces() {
  const int nf = 2 * d, nck = 1 << d;
  // position tolerance: 1e-9 * (1 + max |coordinate|)
  double mx = 0.0;
  for (double v : nodes) mx = std::max(mx, std::fabs(v));
  const double tol = 1e-9 * (1.0 + mx);
  // periodic shifts: c in {-1,0,1}^k, first component slowest, zero skipped
  std::vector<std::vector<double>> shifts;
  int k = n_periodic, total = 1;
  for (int i = 0; i < k; ++i) total *= 3;
  for (int idx = 0; idx < total; ++idx) {
    std::vector<double> v(d, 0.0);
    bool zero = true;
    int rem = idx;
    std::vector<int> c(k);
    for (int i = k - 1; i >= 0; --i) {
      c[i] = rem % 3 - 1;
      rem /= 3;
    }
    for (int i = 0; i < k; ++i) {
      if (c[i]) zero = false;
      for (int j = 0; j < d; ++j) v[j] += c[i] * periodic[i * d + j];
    }
    if (!zero) shifts.push_back(v);
  }
  auto face_corners = [&](int f, int* out) {
    int a = f >> 1, s = f & 1, m = 0;
    for (int c = 0; c < nck; ++c)
      if (((c >> a) & 1) == s) out[m++] = c;
  };
  const int nfc = 1 << (d - 1);
  rface.assign(R * nf, RootFace());
  // exact test of one candidate face, in the rule's order: shared node ids,
  // then each periodic translation
  auto try_match = [&](int64_t r, int f, int64_t r2, int f2, int* corr) -> bool {
    int mine[4], theirs[4];
    face_corners(f, mine);
    face_corners(f2, theirs);
    int64_t a_ids[4], b_ids[4], sa[4], sb[4];
    for (int i = 0; i < nfc; ++i) {
      sa[i] = a_ids[i] = root_corners[r * nck + mine[i]];
      sb[i] = b_ids[i] = root_corners[r2 * nck + theirs[i]];
    }
    std::sort(sa, sa + nfc);
    std::sort(sb, sb + nfc);
    if (std::equal(sa, sa + nfc, sb)) {
      for (int i = 0; i < nfc; ++i)
        for (int j = 0; j < nfc; ++j)
          if (b_ids[j] == a_ids[i]) corr[mine[i]] = theirs[j];
      return true;
    }
    for (const auto& t : shifts) {
      bool ok = true;
      int used[4], nused = 0;
      for (int i = 0; i < nfc && ok; ++i) {
        const double* x = &nodes[a_ids[i] * d];
        int hits = 0, hit = -1;
        for (int j = 0; j < nfc; ++j) {
          const double* y = &nodes[b_ids[j] * d];
          double m = 0.0;
          for (int c = 0; c < d; ++c) m = std::max(m, std::fabs(x[c] + t[c] - y[c]));
          if (m <= tol) {
            ++hits;
            hit = j;
          }
        }
        if (hits != 1 || std::find(used, used + nused, hit) != used + nused) ok = false;
        else {
          used[nused++] = hit;
          corr[mine[i]] = theirs[hit];
        }
      }
      if (ok) return true;
    }
    return false;
  };
  // candidate lookup: faces by sorted corner ids, and by face centre on a
  // grid of cells 8 tol wide.  A face that matches under a translation has
  // its centre within tol of the translated centre, so every face is filed
  // under each cell its tol-box touches and one cell is looked up per shift.
  const double cell = 8.0 * tol;
  auto face_ids = [&](int64_t r, int f) {
    int c[4];
    face_corners(f, c);
    std::vector<int64_t> ids(nfc);
    for (int i = 0; i < nfc; ++i) ids[i] = root_corners[r * nck + c[i]];
    std::sort(ids.begin(), ids.end());
    return ids;
  };
  auto face_centre = [&](int64_t r, int f, double* x) {
    int c[4];
    face_corners(f, c);
    for (int j = 0; j < d; ++j) x[j] = 0.0;
    for (int i = 0; i < nfc; ++i)
      for (int j = 0; j < d; ++j) x[j] += nodes[root_corners[r * nck + c[i]] * d + j] / nfc;
  };
  auto cell_key = [&](const int64_t* q) {
    uint64_t h = 1469598103934665603ull;
    for (int j = 0; j < d; ++j) h = (h ^ (uint64_t)q[j]) * 1099511628211ull;
    return h;
  };
  std::unordered_map<std::string, std::vector<int64_t>> by_ids;
  std::unordered_map<uint64_t, std::vector<int64_t>> by_cell;
  for (int64_t r2 = 0; r2 < R; ++r2)
    for (int f2 = 0; f2 < nf; ++f2) {
      const std::vector<int64_t> ids = face_ids(r2, f2);
      by_ids[std::string((const char*)ids.data(), ids.size() * sizeof(int64_t))].push_back(r2 * nf + f2);
      double x[3];
      face_centre(r2, f2, x);
      int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      for (int j = 0; j < d; ++j) {
        lo[j] = (int64_t)std::floor((x[j] - tol) / cell);
        hi[j] = (int64_t)std::floor((x[j] + tol) / cell);
      }
      for (int o = 0; o < (1 << d); ++o) {
        int64_t q[3] = {0, 0, 0};
        bool dup = false;
        for (int j = 0; j < d; ++j) {
          q[j] = ((o >> j) & 1) ? hi[j] : lo[j];
          if (((o >> j) & 1) && hi[j] == lo[j]) dup = true;
        }
        if (!dup) by_cell[cell_key(q)].push_back(r2 * nf + f2);
      }
    }
  for (int64_t r = 0; r < R; ++r) {
    for (int f = 0; f < nf; ++f) {
      std::vector<int64_t> cand;
      {
        const std::vector<int64_t> ids = face_ids(r, f);
        auto it = by_ids.find(std::string((const char*)ids.data(), ids.size() * sizeof(int64_t)));
        if (it != by_ids.end()) cand.insert(cand.end(), it->second.begin(), it->second.end());
      }
      double x[3];
      face_centre(r, f, x);
      for (const auto& t : shifts) {
        int64_t q[3] = {0, 0, 0};
        for (int j = 0; j < d; ++j) q[j] = (int64_t)std::floor((x[j] + t[j]) / cell);
        auto it = by_cell.find(cell_key(q));
        if (it != by_cell.end()) cand.insert(cand.end(), it->second.begin(), it->second.end());
      }
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      // the first face in (root, face) order that passes the exact test
      bool found = false;
      int corr[8];
      int64_t r2f = -1;
      int f2f = -1;
      for (int64_t code : cand) {
        const int64_t r2 = code / nf;
        const int f2 = (int)(code % nf);
        if (r2 == r && f2 == f) continue;
        if (try_match(r, f, r2, f2, corr)) {
          found = true;
          r2f = r2;
          f2f = f2;
          break;
        }
      }
      int mine[4];
      face_corners(f, mine);
      if (!found) continue;
      // orientation from the corner correspondence
      RootFace rf;
      rf.valid = true;
      rf.root = r2f;
      rf.face = f2f;
      int a = f >> 1, s = f & 1, b2 = f2f >> 1, s2 = f2f & 1;
      rf.o.pi[a] = b2;
      rf.o.sg[a] = (s != s2) ? 1 : -1;
      int base = s << a;  // all tangential bits zero
      for (int t = 0; t < d; ++t) {
        if (t == a) continue;
        int other = base | (1 << t);
        int kb = corr[base], ko = corr[other];
        int diff = kb ^ ko;
        int ax = -1;
        for (int u = 0; u < d; ++u)
          if (diff == (1 << u)) ax = u;
        if (ax < 0 || ax == b2) return error = "root faces do not match as a hexahedral face", false;
        rf.o.pi[t] = ax;
        rf.o.sg[t] = ((ko >> ax) & 1) ? 1 : -1;
      }
      // verify every corner
      for (int i = 0; i < nfc; ++i) {
        int kc = mine[i], k2 = corr[kc];
        for (int t = 0; t < d; ++t) {
          if (t == a) continue;
          int bit = (kc >> t) & 1;
          int want = rf.o.sg[t] > 0 ? bit : 1 - bit;
          if (((k2 >> rf.o.pi[t]) & 1) != want) return error = "inconsistent root face corners", false;
        }
      }
      rface[r * nf + f] = rf;
    }
  }
  return true;
}

// ------------------------------------------------------------------- tree
bool Forest::neighbour(int64_t root, int level, const int* pos, int f, int64_t* root2, int* q,
                       Orient* o, int* f2) const {
  const int a = f >> 1, s = f & 1;
  const int L = 1 << (level - 1);
  int p2[3] = {pos[0], pos[1], pos[2]};
  p2[a] += s ? 1 : -1;
  if (p2[a] >= 0 && p2[a] < L) {
    *root2 = root;
    for (int u = 0; u < 3; ++u) q[u] = p2[u];
    *o = Orient();
    *f2 = 2 * a + (1 - s);
    return true;
  }
  const RootFace& rf = rface[root * 2 * d + f];
  if (!rf.valid) return false;
  int qq[3] = {0, 0, 0};
  for (int t = 0; t < d; ++t) {
    if (t == a) continue;
    qq[rf.o.pi[t]] = rf.o.sg[t] > 0 ? pos[t] : L - 1 - pos[t];
  }
  const int b2 = rf.face >> 1, s2 = rf.face & 1;
  qq[b2] = s2 == 0 ? 0 : L - 1;
  *root2 = rf.root;
  for (int u = 0; u < 3; ++u) q[u] = qq[u];
  *o = rf.o;
  *f2 = rf.face;
  return true;
}

void Forest::collect(uint64_t k, std::vector<uint64_t>& out) const {
  auto it = tree.find(k);
  if (it->second) {
    out.push_back(k);
    return;
  }
  int64_t r;
  int lev, pos[3];
  unkey(k, &r, &lev, pos);
  for (int c = 0; c < (1 << d); ++c) {
    int cp[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) cp[a] = 2 * pos[a] + ((c >> a) & 1);
    collect(key(r, lev + 1, cp), out);
  }
}

void Forest::order_leaves() {
  leaves.clear();
  int z[3] = {0, 0, 0};
  for (int64_t r = 0; r < R; ++r) collect(key(r, 1, z), leaves);
  leaf_index.clear();
  for (size_t i = 0; i < leaves.size(); ++i) leaf_index[leaves[i]] = (int64_t)i;
}

void Forest::refine_key(uint64_t k) {
  int64_t r;
  int lev, pos[3];
  unkey(k, &r, &lev, pos);
  tree[k] = 0;
  for (int c = 0; c < (1 << d); ++c) {
    int cp[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) cp[a] = 2 * pos[a] + ((c >> a) & 1);
    tree[key(r, lev + 1, cp)] = 1;
  }
}

bool Forest::find_containing_leaf(int64_t root, int level, const int* pos, uint64_t* out,
                                  int* out_level) const {
  for (int l = level; l >= 1; --l) {
    int pp[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) pp[a] = pos[a] >> (level - l);
    auto it = tree.find(key(root, l, pp));
    if (it == tree.end()) continue;
    if (!it->second) return false;
    *out = it->first;
    *out_level = l;
    return true;
  }
  return false;
}

std::vector<uint64_t> Forest::violations() const {
  std::vector<uint64_t> out;
  for (uint64_t k : leaves) {
    int64_t r;
    int lev, pos[3];
    unkey(k, &r, &lev, pos);
    for (int f = 0; f < 2 * d; ++f) {
      int64_t r2;
      int q[3], f2;
      Orient o;
      if (!neighbour(r, lev, pos, f, &r2, q, &o, &f2)) continue;
      if (tree.count(key(r2, lev, q))) continue;
      uint64_t c;
      int cl;
      if (find_containing_leaf(r2, lev, q, &c, &cl) && cl < lev - 1) out.push_back(c);
    }
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

bool Forest::refine(const std::vector<uint64_t>& keys) {
  for (uint64_t k : keys) {
    auto it = tree.find(k);
    if (it == tree.end() || !it->second) return error = "refine: not a leaf", false;
    int64_t r;
    int lev, pos[3];
    unkey(k, &r, &lev, pos);
    if (lev >= 12) return error = "refine: level limit (12) reached", false;
  }
  for (uint64_t k : keys)
    if (tree[k]) refine_key(k);
  order_leaves();
  for (;;) {
    std::vector<uint64_t> v = violations();
    if (v.empty()) break;
    for (uint64_t k : v)
      if (tree[k]) refine_key(k);
    order_leaves();
  }
  return true;
}

bool Forest::coarsen(const std::vector<uint64_t>& parents, bool* balance_violation) {
  *balance_violation = false;
  auto saved = tree;
  for (uint64_t k : parents) {
    auto it = tree.find(k);
    int64_t r;
    int lev, pos[3];
    unkey(k, &r, &lev, pos);
    bool ok = it != tree.end() && it->second == 0;
    std::vector<uint64_t> kids;
    for (int c = 0; ok && c < (1 << d); ++c) {
      int cp[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cp[a] = 2 * pos[a] + ((c >> a) & 1);
      uint64_t ck = key(r, lev + 1, cp);
      auto jt = tree.find(ck);
      if (jt == tree.end() || !jt->second) ok = false;
      kids.push_back(ck);
    }
    if (!ok) {
      tree = saved;
      order_leaves();
      *balance_violation = true;
      return error = "coarsen: children are not all leaves", false;
    }
    for (uint64_t ck : kids) tree.erase(ck);
    tree[k] = 1;
  }
  order_leaves();
  if (!violations().empty()) {
    tree = saved;
    order_leaves();
    *balance_violation = true;
    return error = "coarsen would break 2:1 balance", false;
  }
  return true;
}

bool Forest::can_coarsen(uint64_t parent) const {
  auto it = tree.find(parent);
  if (it == tree.end() || it->second) return false;
  int64_t r;
  int lev, pos[3];
  unkey(parent, &r, &lev, pos);
  for (int c = 0; c < (1 << d); ++c) {
    int cp[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) cp[a] = 2 * pos[a] + ((c >> a) & 1);
    auto jt = tree.find(key(r, lev + 1, cp));
    if (jt == tree.end() || !jt->second) return false;
  }
  // a face neighbour region at the parent's level that is refined, with a
  // refined child on the shared face, holds leaves two levels finer
  for (int f = 0; f < 2 * d; ++f) {
    int64_t r2;
    int q[3], f2;
    Orient o;
    if (!neighbour(r, lev, pos, f, &r2, q, &o, &f2)) continue;
    auto nt = tree.find(key(r2, lev, q));
    if (nt == tree.end() || nt->second) continue;
    const int b2 = f2 >> 1, s2 = f2 & 1;
    for (int c = 0; c < (1 << d); ++c) {
      if (((c >> b2) & 1) != s2) continue;
      int cp[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cp[a] = 2 * q[a] + ((c >> a) & 1);
      auto ct = tree.find(key(r2, lev + 1, cp));
      if (ct != tree.end() && !ct->second) return false;
    }
  }
  return true;
}

int64_t Forest::adapt(const std::vector<uint64_t>& refine_keys, const std::vector<uint64_t>& low_sorted) {
  if (!refine_keys.empty()) refine(refine_keys);
  const std::vector<uint64_t> snapshot = leaves;
  int64_t n = 0;
  for (uint64_t k : snapshot) {
    int64_t r;
    int lev, pos[3];
    unkey(k, &r, &lev, pos);
    bool first = lev > 1;
    for (int a = 0; a < d; ++a) first = first && (pos[a] & 1) == 0;
    if (!first) continue;
    auto it = tree.find(k);
    if (it == tree.end() || !it->second) continue;
    int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
    const uint64_t parent = key(r, lev - 1, pp);
    bool low = true;
    for (int c = 0; c < (1 << d) && low; ++c) {
      int cp[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cp[a] = 2 * pp[a] + ((c >> a) & 1);
      low = std::binary_search(low_sorted.begin(), low_sorted.end(), key(r, lev, cp));
    }
    if (!low || !can_coarsen(parent)) continue;
    for (int c = 0; c < (1 << d); ++c) {
      int cp[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cp[a] = 2 * pp[a] + ((c >> a) & 1);
      tree.erase(key(r, lev, cp));
    }
    tree[parent] = 1;
    ++n;
  }
  order_leaves();
  return n;
}

Forest::Tables Forest::tables() const {
  Tables T;
  const int64_t L = n_leaves();
  const int nf = 2 * d;
  T.root.assign(L, 0);
  T.level.assign(L, 0);
  T.pos.assign(L * d, 0);
  T.kind.assign(L * nf, 0);
  T.orient.assign(L * nf, 0);
  T.nbr.assign(L * nf * 4, -1);
  for (int64_t i = 0; i < L; ++i) {
    int64_t r;
    int lev, pos[3];
    unkey(leaves[i], &r, &lev, pos);
    T.root[i] = (int32_t)r;
    T.level[i] = lev;
    for (int a = 0; a < d; ++a) T.pos[i * d + a] = pos[a];
    for (int f = 0; f < nf; ++f) {
      int64_t r2;
      int q[3], f2;
      Orient o;
      if (!neighbour(r, lev, pos, f, &r2, q, &o, &f2)) {
        T.kind[i * nf + f] = kBoundary;
        continue;
      }
      T.orient[i * nf + f] = orient_code(o, d);
      auto it = tree.find(key(r2, lev, q));
      if (it != tree.end() && it->second) {
        T.kind[i * nf + f] = kSame;
        T.nbr[(i * nf + f) * 4] = leaf_index.at(it->first);
      } else if (it != tree.end()) {
        T.kind[i * nf + f] = kFiner;
        const int a = f >> 1, b2 = f2 >> 1, s2 = f2 & 1;
        for (int sub = 0; sub < (1 << (d - 1)); ++sub) {
          int cc[3] = {0, 0, 0}, j = 0;
          for (int t = 0; t < d; ++t) {
            if (t == a) continue;
            int bit = (sub >> j) & 1;
            cc[o.pi[t]] = o.sg[t] > 0 ? bit : 1 - bit;
            ++j;
          }
          cc[b2] = s2 == 0 ? 0 : 1;
          int cp[3] = {0, 0, 0};
          for (int u = 0; u < d; ++u) cp[u] = 2 * q[u] + cc[u];
          T.nbr[(i * nf + f) * 4 + sub] = leaf_index.at(key(r2, lev + 1, cp));
        }
      } else {
        T.kind[i * nf + f] = kCoarser;
        int cp[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
        T.nbr[(i * nf + f) * 4] = leaf_index.at(key(r2, lev - 1, cp));
      }
    }
  }
  return T;
}

// --------------------------------------------------------------- geometry
// nodes of a child block from its parent's nodes: each child node is the
// parent's (bi/tri)linear interpolant at the child node's position
static void child_nodes(int d, int n, const int* pos, const std::vector<double>& PX, std::vector<double>& out) {
  const int nn1 = n + 1;
  const int nn = (int)std::pow(nn1, d);
  out.assign((size_t)nn * d, 0.0);
  for (int li = 0; li < nn; ++li) {
    int I[3] = {0, 0, 0}, t = li;
    for (int a = 0; a < d; ++a) {
      I[a] = t % nn1;
      t /= nn1;
    }
    int Pc[3] = {0, 0, 0};
    double xi[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      int H = (pos[a] & 1) * n + I[a];
      Pc[a] = std::min(H / 2, n - 1);
      xi[a] = (double)(H - 2 * Pc[a] - 1);
    }
    for (int c = 0; c < (1 << d); ++c) {
      double wgt = 1.0;
      int J = 0, stride = 1;
      for (int a = 0; a < d; ++a) {
        int bit = (c >> a) & 1;
        wgt *= 0.5 * (1.0 + (bit ? 1.0 : -1.0) * xi[a]);
        J += (Pc[a] + bit) * stride;
        stride *= nn1;
      }
      if (wgt == 0.0) continue;
      for (int j = 0; j < d; ++j) out[li * d + j] += wgt * PX[J * d + j];
    }
  }
}

const std::vector<double>& Forest::block_nodes(uint64_t k) {
  auto it = node_cache_.find(k);
  if (it != node_cache_.end()) return it->second;
  int64_t r;
  int lev, pos[3];
  unkey(k, &r, &lev, pos);
  if (lev == 1) return node_cache_[k] = root_nodes[r];
  int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
  const std::vector<double> PX = block_nodes(key(r, lev - 1, pp));  // copy: the cache may rehash
  std::vector<double> out;
  child_nodes(d, n, pos, PX, out);
  return node_cache_[k] = std::move(out);
}

std::vector<uint64_t> Forest::uncached_nodes(const std::vector<uint64_t>& keys) const {
  std::vector<uint64_t> out;
  std::unordered_set<uint64_t> seen;
  for (uint64_t k : keys) {
    // walk up until a cached block (or a root)
    while (!node_cache_.count(k) && seen.insert(k).second) {
      out.push_back(k);
      int64_t r;
      int lev, pos[3];
      unkey(k, &r, &lev, pos);
      if (lev == 1) break;
      int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
      k = key(r, lev - 1, pp);
    }
  }
  auto level_of = [](uint64_t k) {
    int64_t r;
    int lev, pos[3];
    unkey(k, &r, &lev, pos);
    return lev;
  };
  std::stable_sort(out.begin(), out.end(), [&](uint64_t a, uint64_t b) { return level_of(a) < level_of(b); });
  return out;
}

void Forest::compute_nodes(uint64_t k, std::vector<double>& out) const {
  int64_t r;
  int lev, pos[3];
  unkey(k, &r, &lev, pos);
  if (lev == 1) {
    out = root_nodes[r];
    return;
  }
  int pp[3] = {pos[0] >> 1, pos[1] >> 1, pos[2] >> 1};
  child_nodes(d, n, pos, node_cache_.at(key(r, lev - 1, pp)), out);
}

void Forest::cell_coefficients(uint64_t k, std::vector<double>& out) {
  const std::vector<double>& X = node_cache_.count(k) ? node_cache_.at(k) : block_nodes(k);
  const int nc = (int)std::pow(n, d), nn1 = n + 1, ncor = 1 << d;
  // sign of corner kap in the coefficient of monomial c: prod over a in c of (+-1)
  double sgn[8][8];
  for (int c = 0; c < ncor; ++c)
    for (int kap = 0; kap < ncor; ++kap) {
      double s = 1.0;
      for (int a = 0; a < d; ++a)
        if ((c >> a) & 1) s *= ((kap >> a) & 1) ? 1.0 : -1.0;
      sgn[c][kap] = s;
    }
  out.assign((size_t)ncor * d * nc, 0.0);
  for (int cell = 0; cell < nc; ++cell) {
    int I[3] = {0, 0, 0}, t = cell;
    for (int a = 0; a < d; ++a) {
      I[a] = t % n;
      t /= n;
    }
    double xk[8][3];
    for (int kap = 0; kap < ncor; ++kap) {
      int J = 0, stride = 1;
      for (int a = 0; a < d; ++a) {
        J += (I[a] + ((kap >> a) & 1)) * stride;
        stride *= nn1;
      }
      for (int j = 0; j < d; ++j) xk[kap][j] = X[J * d + j];
    }
    for (int c = 0; c < ncor; ++c)
      for (int j = 0; j < d; ++j) {
        double acc = 0.0;
        for (int kap = 0; kap < ncor; ++kap) acc += sgn[c][kap] * xk[kap][j] / ncor;
        out[((size_t)c * d + j) * nc + cell] = acc;
      }
  }
}

void eval_map(int d, const double* coef, const double* xi, double* x, double* A) {
  // coef[c*d + j]; x(xi) = sum_c X_c prod_{a in c} xi_a
  const int ncor = 1 << d;
  for (int j = 0; j < d; ++j) {
    if (x) x[j] = 0.0;
    for (int a = 0; a < d; ++a) A[j * d + a] = 0.0;
  }
  for (int c = 0; c < ncor; ++c) {
    double mono = 1.0;
    for (int a = 0; a < d; ++a)
      if ((c >> a) & 1) mono *= xi[a];
    for (int j = 0; j < d; ++j)
      if (x) x[j] += coef[c * d + j] * mono;
    for (int a = 0; a < d; ++a) {
      if (!((c >> a) & 1)) continue;
      double m = 1.0;
      for (int b = 0; b < d; ++b)
        if (b != a && ((c >> b) & 1)) m *= xi[b];
      for (int j = 0; j < d; ++j) A[j * d + a] += coef[c * d + j] * m;
    }
  }
}

double det_and_cofactor(int d, const double* A, double* Ja) {
  // A[j*d+a] = dx_j/dxi_a; Ja[i*d+j] = J dxi_i/dx_j (rows = cross products)
  if (d == 2) {
    double xs = A[0], xe = A[1], ys = A[2], ye = A[3];
    Ja[0] = ye;
    Ja[1] = -xe;
    Ja[2] = -ys;
    Ja[3] = xs;
    return xs * ye - xe * ys;
  }
  double c[3][3];  // columns: c[a][j] = dx_j/dxi_a
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 3; ++j) c[a][j] = A[j * 3 + a];
  for (int i = 0; i < 3; ++i) {
    const double* u = c[(i + 1) % 3];
    const double* v = c[(i + 2) % 3];
    Ja[i * 3 + 0] = u[1] * v[2] - u[2] * v[1];
    Ja[i * 3 + 1] = u[2] * v[0] - u[0] * v[2];
    Ja[i * 3 + 2] = u[0] * v[1] - u[1] * v[0];
  }
  return c[0][0] * Ja[0] + c[0][1] * Ja[1] + c[0][2] * Ja[2];
}

}  // namespace dgf
