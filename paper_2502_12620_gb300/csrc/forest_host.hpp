// Host-side block forest: topology, refinement, integer leaf tables, FP64
// geometry and the FP64 operators the kernels consume.
//
// Sec. 3.1: quad/oct trees grown from unstructured root blocks (roots at
// level 1), neighbours of new blocks follow from the parent's neighbours and
// the position among siblings, R records relative rotations.
// Sec. 3.3, Eq. (6): block cell nodes by (bi/tri)linear interpolation;
// children's nodes by the same interpolation of the parent's cells.
// Sec. 3.4, Eqs. (13)-(14): the combine operator, assembled here in FP64.
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace dgf {

constexpr int kSame = 0, kCoarser = 1, kFiner = 2, kBoundary = 3;

// Signed axis permutation: my axis a -> neighbour axis pi[a], sign sg[a].
struct Orient {
  int pi[3] = {0, 1, 2};
  int sg[3] = {1, 1, 1};
};

int orient_code(const Orient& o, int d);
Orient orient_from_code(int code, int d);

// Reference-element tables of degree p (FP64), built from Gauss-Legendre
// nodes found by Newton iteration on P_N.
struct Basis1D {
  int N = 0;
  std::vector<double> x, w;   // nodes, weights
  std::vector<double> V;      // V[q*N+k]  = P_k(x_q)
  std::vector<double> Vi;     // Vi[k*N+q] = (2k+1)/2 w_q P_k(x_q)  (= V^{-1})
  std::vector<double> Dn;     // Dn[q*N+j] = l_j'(x_q) (nodal derivative)
  std::vector<double> Sh;     // Sh[q*N+j] = (w_j/w_q) Dn[j*N+q] (weak form)
  std::vector<double> lp, lm; // l_q(+1), l_q(-1)
  std::vector<double> Sm, Sp; // split: S[l*N+k] coefficients of P_k((xi-+1)/2)
  std::vector<double> Snm, Snp;  // nodal split: Sn[i*N+j] = l_j((x_i -+ 1)/2)
  double lagrange(int j, double xi) const;  // l_j(xi) of the Gauss points
  void build(int N);
};
double legendre(int k, double x);
double legendre_deriv(int k, double x);

class Forest {
 public:
  int d = 0, n = 0, p = 0;
  std::vector<double> nodes;             // n_nodes * d
  std::vector<int64_t> root_corners;     // R * 2^d
  std::vector<std::vector<double>> root_nodes;  // (n+1)^d * d per root
  std::vector<double> periodic;          // k * d
  int n_periodic = 0;
  int64_t R = 0;

  struct RootFace {
    bool valid = false;
    int64_t root = -1;
    int face = -1;
    Orient o;
  };
  std::vector<RootFace> rface;  // R * 2d

  // tree: key -> 1 leaf / 0 internal
  std::unordered_map<uint64_t, uint8_t> tree;
  std::vector<uint64_t> leaves;  // canonical order
  std::unordered_map<uint64_t, int64_t> leaf_index;

  std::string error;

  static uint64_t key(int64_t root, int level, const int* pos);
  static void unkey(uint64_t k, int64_t* root, int* level, int* pos);

  // returns false with `error` set on a malformed description
  bool init(int dim, int n_seg, int deg, int64_t n_nodes, const double* xyz, int64_t n_roots,
            const int64_t* corners, const double* cell_nodes, int n_per, const double* per);

  // same-level block across face f; false at a domain boundary
  bool neighbour(int64_t root, int level, const int* pos, int f, int64_t* root2, int* q,
                 Orient* o, int* f2) const;

  // refine leaves (by key) and close under 2:1 face balance
  bool refine(const std::vector<uint64_t>& keys);
  // coarsen parents; false (unchanged) with error on violation
  bool coarsen(const std::vector<uint64_t>& parents, bool* balance_violation);
  // one adaptation pass (refine the given leaves with closure, then visit
  // the leaves in canonical order and coarsen each sibling group whose
  // members all satisfy low(key) where balance allows); returns the number
  // of parents coarsened
  int64_t adapt(const std::vector<uint64_t>& refine_keys, const std::vector<uint64_t>& low_sorted);

  void order_leaves();
  int64_t n_leaves() const { return (int64_t)leaves.size(); }

  struct Tables {
    std::vector<int32_t> root, level, pos, kind, orient;
    std::vector<int64_t> nbr;
  };
  Tables tables() const;

  // geometry
  const std::vector<double>& block_nodes(uint64_t k);
  // Filling the node cache for many blocks from several threads: the blocks
  // (and their ancestors) whose nodes are not cached, in increasing level
  // order; the nodes of one of them from its parent's cached nodes (reads
  // the cache only, so blocks of one level may run concurrently); and the
  // insertion of the result (one thread).
  std::vector<uint64_t> uncached_nodes(const std::vector<uint64_t>& keys) const;
  void compute_nodes(uint64_t k, std::vector<double>& out) const;
  void put_nodes(uint64_t k, std::vector<double>&& X) { node_cache_[k] = std::move(X); }
  // trilinear coefficients X_c (c = 0..2^d-1, c = variable mask) of every
  // cell of a leaf: out[(c*d + j)*nc + cell]
  void cell_coefficients(uint64_t k, std::vector<double>& out);

 private:
  std::unordered_map<uint64_t, std::vector<double>> node_cache_;
  bool match_root_faces();
  void refine_key(uint64_t k);
  void collect(uint64_t k, std::vector<uint64_t>& out) const;
  bool find_containing_leaf(int64_t root, int level, const int* pos, uint64_t* out,
                            int* out_level) const;
  std::vector<uint64_t> violations() const;
  // parent's children are all leaves and making it a leaf keeps 2:1 face
  // balance (no leaf two levels finer would touch it)
  bool can_coarsen(uint64_t parent) const;
};

// x(xi), dx/dxi and (J, J dxi_i/dx_j) from trilinear coefficients of one
// cell (coef[(c*d+j)] layout for a single cell).
void eval_map(int d, const double* coef, const double* xi, double* x, double* A);
double det_and_cofactor(int d, const double* A, double* Ja);

}  // namespace dgf
