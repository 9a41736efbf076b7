// Host set-up of the decomposition (Sec. 1, eq. NumberFive) and of the
// face-local interface preconditioner (Sec. 3, eq. NumberEight/NumberNine,
// with the cross points removed as in Sec. 4).  Pure C++, runs once per
// geometry.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "ddel_internal.h"
#include "ddel_globalprec.h"

namespace ddel {

namespace {

// Local node order of the reference element: (0,0),(1,0),(1,1),(0,1) and the
// same four again at z = 1 in 3D.
const int kRef2[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};

void ref_offsets(int dim, int a, int off[3]) {
  off[0] = kRef2[a & 3][0];
  off[1] = kRef2[a & 3][1];
  off[2] = dim == 3 ? (a >> 2) : 0;
}

}  // namespace

void element_stiffness(int dim, double nu, int plane_stress, std::vector<double>* Ke) {
  // Voigt elasticity matrix for E = 1 from the Lame constants of Sec. 1.
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const int nv = dim == 2 ? 3 : 6;
  double D[6][6] = {};
  if (dim == 2) {
    if (plane_stress) lam = 2.0 * mu * lam / (lam + 2.0 * mu);
    D[0][0] = D[1][1] = lam + 2 * mu;
    D[0][1] = D[1][0] = lam;
    D[2][2] = mu;
  } else {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) D[i][j] = lam + (i == j ? 2 * mu : 0.0);
    D[3][3] = D[4][4] = D[5][5] = mu;
  }
  const int nnode = 1 << dim, nd = dim * nnode;
  Ke->assign(nd * nd, 0.0);
  const double g = 1.0 / std::sqrt(3.0);  // 2-point Gauss on [-1, 1]
  const int nq = 1 << dim;
  for (int q = 0; q < nq; ++q) {
    double xi[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
    // derivatives of the multilinear shape functions; unit element: d/dx = 2 d/dxi
    double dN[8][3];
    for (int a = 0; a < nnode; ++a) {
      int off[3];
      ref_offsets(dim, a, off);
      for (int k = 0; k < dim; ++k) {
        double v = (2 * off[k] - 1) * 0.5;
        for (int m = 0; m < dim; ++m)
          if (m != k) v *= 0.5 * (1.0 + (2 * off[m] - 1) * xi[m]);
        dN[a][k] = 2.0 * v;
      }
    }
    double B[6][24] = {};
    for (int a = 0; a < nnode; ++a) {
      if (dim == 2) {
        B[0][2 * a] = dN[a][0];
        B[1][2 * a + 1] = dN[a][1];
        B[2][2 * a] = dN[a][1];
        B[2][2 * a + 1] = dN[a][0];
      } else {
        const int c = 3 * a;
        B[0][c] = dN[a][0];
        B[1][c + 1] = dN[a][1];
        B[2][c + 2] = dN[a][2];
        B[3][c] = dN[a][1];
        B[3][c + 1] = dN[a][0];
        B[4][c + 1] = dN[a][2];
        B[4][c + 2] = dN[a][1];
        B[5][c] = dN[a][2];
        B[5][c + 2] = dN[a][0];
      }
    }
    const double w = std::pow(0.5, dim);  // weight 1 per point times Jacobian (1/2)^dim
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) {
        double s = 0.0;
        for (int p = 0; p < nv; ++p) {
          double dp = 0.0;
          for (int r = 0; r < nv; ++r) dp += D[p][r] * B[r][j];
          s += B[p][i] * dp;
        }
        (*Ke)[i * nd + j] += w * s;
      }
  }
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j < i; ++j) {
      double s = 0.5 * ((*Ke)[i * nd + j] + (*Ke)[j * nd + i]);
      (*Ke)[i * nd + j] = (*Ke)[j * nd + i] = s;
    }
}

bool gen_eig(int n, const std::vector<double>& L, const std::vector<double>& M,
             std::vector<double>* mu, std::vector<double>* V) {
  // M = R R^T (Cholesky, lower R)
  std::vector<double> R(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = M[j * n + j];
    for (int k = 0; k < j; ++k) d -= R[j * n + k] * R[j * n + k];
    if (!(d > 0)) return false;
    R[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = M[i * n + j];
      for (int k = 0; k < j; ++k) s -= R[i * n + k] * R[j * n + k];
      R[i * n + j] = s / R[j * n + j];
    }
  }
  auto fwd = [&](std::vector<double>& X) {  // X <- R^-1 X (columns)
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < n; ++i) {
        double s = X[i * n + c];
        for (int k = 0; k < i; ++k) s -= R[i * n + k] * X[k * n + c];
        X[i * n + c] = s / R[i * n + i];
      }
  };
  std::vector<double> A = L;
  fwd(A);  // R^-1 L
  std::vector<double> T(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[i * n + j] = A[j * n + i];
  fwd(T);  // R^-1 (R^-1 L)^T = R^-1 L R^-T
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      double s = 0.5 * (T[i * n + j] + T[j * n + i]);
      T[i * n + j] = T[j * n + i] = s;
    }
  // cyclic Jacobi rotations on T, accumulating Q
  std::vector<double> Q(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += T[i * n + j] * T[i * n + j];
        if (i != j) off += T[i * n + j] * T[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = T[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = T[p * n + p], aqq = T[q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = T[k * n + p], akq = T[k * n + q];
          T[k * n + p] = c * akp - s * akq;
          T[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = T[p * n + k], aqk = T[q * n + k];
          T[p * n + k] = c * apk - s * aqk;
          T[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  // sort eigenvalues ascending
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return T[a * n + a] < T[b * n + b]; });
  mu->resize(n);
  V->assign(n * n, 0.0);
  // V = R^-T Q: back substitution R^T v = q per column
  for (int jj = 0; jj < n; ++jj) {
    const int j = ord[jj];
    (*mu)[jj] = T[j * n + j];
    for (int i = n - 1; i >= 0; --i) {
      double s = Q[i * n + j];
      for (int k = i + 1; k < n; ++k) s -= R[k * n + i] * (*V)[k * n + jj];
      (*V)[i * n + jj] = s / R[i * n + i];
    }
  }
  return true;
}

std::string build_setup(int dim, const int ne_in[3], int sub, double E, double nu,
                        int plane_stress, uint32_t clamp_faces, const uint8_t* fixed_dof,
                        int n_point, const int64_t* point_node, const double* point_force,
                        int traction_face, const double traction[3], const double body_force[3],
                        double theta, Setup* S) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5)) return "need E > 0 and -1 < nu < 1/2";
  if (sub < 1) return "sub must be positive";
  if (!(theta >= 0.0 && theta <= 1.0)) return "theta must lie in [0, 1]";
  S->dim = dim;
  S->sub = sub;
  for (int a = 0; a < 3; ++a) {
    S->ne[a] = a < dim ? ne_in[a] : 0;
    if (a < dim && (S->ne[a] < 1 || S->ne[a] % sub)) return "sub must divide every grid size";
    S->nn[a] = a < dim ? S->ne[a] + 1 : 1;
    S->nsa[a] = a < dim ? S->ne[a] / sub : 1;
  }
  S->n_sub = S->nsa[0] * S->nsa[1] * S->nsa[2];
  S->n_nodes = (int64_t)S->nn[0] * S->nn[1] * S->nn[2];
  S->n_dof = dim * S->n_nodes;
  S->n_elem = (int64_t)S->ne[0] * S->ne[1] * (dim == 3 ? S->ne[2] : 1);
  if (S->n_dof > (int64_t)1 << 31) return "grid too large for 32-bit DOF tables";
  const int s = sub;
  const int64_t nn1 = S->nn[1], nn2 = S->nn[2];
  auto node_of = [&](int i, int j, int k) -> int64_t { return ((int64_t)i * nn1 + j) * nn2 + k; };

  element_stiffness(dim, nu, plane_stress, &S->Ke);
  for (auto& v : S->Ke) v *= 1.0;  // unit E: scaled per element by E rho^p

  // ---- boundary conditions and loads --------------------------------------
  S->fixed.assign(S->n_dof, 0);
  S->f.assign(S->n_dof, 0.0);
  if (fixed_dof)
    for (int64_t d = 0; d < S->n_dof; ++d) S->fixed[d] = fixed_dof[d] ? 1 : 0;
  for (int a = 0; a < dim; ++a)
    for (int side = 0; side < 2; ++side) {
      if (!(clamp_faces & (1u << (2 * a + side)))) continue;
      const int val = side ? S->ne[a] : 0;
      for (int i = 0; i < S->nn[0]; ++i)
        for (int j = 0; j < S->nn[1]; ++j)
          for (int k = 0; k < S->nn[2]; ++k) {
            const int c[3] = {i, j, k};
            if (c[a] != val) continue;
            const int64_t n = node_of(i, j, k);
            for (int comp = 0; comp < dim; ++comp) S->fixed[dim * n + comp] = 1;
          }
    }
  for (int p = 0; p < n_point; ++p) {
    const int64_t n = point_node[p];
    if (n < 0 || n >= S->n_nodes) return "point load node out of range";
    for (int comp = 0; comp < dim; ++comp) S->f[dim * n + comp] += point_force[dim * p + comp];
  }
  if (traction_face >= 0) {
    const int a = traction_face / 2, side = traction_face % 2;
    if (a >= dim) return "traction face out of range";
    const int val = side ? S->ne[a] : 0;
    const int t1 = (a + 1) % dim, t2 = (a + 2) % dim;
    const double share = dim == 2 ? 0.5 : 0.25;
    const int n1 = S->ne[t1], n2 = dim == 3 ? S->ne[t2] : 1;
    for (int u = 0; u < n1; ++u)
      for (int v = 0; v < n2; ++v)
        for (int cu = 0; cu < 2; ++cu)
          for (int cv = 0; cv < (dim == 3 ? 2 : 1); ++cv) {
            int c[3] = {0, 0, 0};
            c[a] = val;
            c[t1] = u + cu;
            if (dim == 3) c[t2] = v + cv;
            const int64_t n = node_of(c[0], c[1], c[2]);
            for (int comp = 0; comp < dim; ++comp) S->f[dim * n + comp] += share * traction[comp];
          }
  }
  if (body_force && (body_force[0] != 0.0 || body_force[1] != 0.0 || (dim == 3 && body_force[2] != 0.0))) {
    // consistent loads of a uniform body force: every unit element gives
    // 1/2^dim of its force to each of its nodes
    const double share = dim == 2 ? 0.25 : 0.125;
    for (int i = 0; i < S->ne[0]; ++i)
      for (int j = 0; j < S->ne[1]; ++j)
        for (int k = 0; k < (dim == 3 ? S->ne[2] : 1); ++k)
          for (int dx = 0; dx < 2; ++dx)
            for (int dy = 0; dy < 2; ++dy)
              for (int dz = 0; dz < (dim == 3 ? 2 : 1); ++dz) {
                const int64_t n = node_of(i + dx, j + dy, k + dz);
                for (int comp = 0; comp < dim; ++comp) S->f[dim * n + comp] += share * body_force[comp];
              }
  }
  for (int64_t d = 0; d < S->n_dof; ++d)
    if (S->fixed[d]) S->f[d] = 0.0;

  // ---- Gamma classification (reading: a node is on Gamma iff it lies in the
  // closure of two or more subdomains) --------------------------------------
  auto cnt = [&](int a, int x) { return (x % s == 0 && x > 0 && x < S->ne[a]) ? 2 : 1; };
  auto node_mult = [&](int i, int j, int k) {
    int m = cnt(0, i) * cnt(1, j);
    if (dim == 3) m *= cnt(2, k);
    return m;
  };
  std::vector<int64_t> cross_dofs;
  // faces: key (normal axis, plane, q of the tangential axes) -> nodes
  std::map<std::tuple<int, int, int, int>, std::vector<int64_t>> faces;
  for (int i = 0; i < S->nn[0]; ++i)
    for (int j = 0; j < S->nn[1]; ++j)
      for (int k = 0; k < S->nn[2]; ++k) {
        const int m = node_mult(i, j, k);
        if (m < 2) continue;
        const int64_t n = node_of(i, j, k);
        if (m > 2) {
          for (int comp = 0; comp < dim; ++comp)
            if (!S->fixed[dim * n + comp]) cross_dofs.push_back(dim * n + comp);
          continue;
        }
        const int c[3] = {i, j, k};
        int na = 0;
        for (int a = 0; a < dim; ++a)
          if (cnt(a, c[a]) == 2) na = a;
        int q[2] = {0, 0}, qi = 0;
        for (int a = 0; a < dim; ++a) {
          if (a == na) continue;
          q[qi++] = c[a] == S->ne[a] ? S->nsa[a] - 1 : c[a] / s;
        }
        faces[std::make_tuple(na, c[na] / s, q[0], q[1])].push_back(n);
      }

  // ---- face blocks: assemble M, L on the face patch, restrict, invert -------
  // 1D P1 element matrices on unit edges; the 2D Q1 ones on unit squares are
  // their Kronecker sums: M2 = M1 (x) M1, L2 = L1 (x) M1 + M1 (x) L1.
  const double M1[2][2] = {{2.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 6}};
  const double L1[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
  S->gamma_dof.clear();
  S->blk_off.clear();
  S->blk_n.clear();
  S->blk_poff.clear();
  S->blk_hmean.clear();
  S->ptab.clear();
  std::map<std::vector<double>, std::pair<int, double>> pcache;  // key -> (poff, hmean)
  std::map<std::vector<double>, std::vector<double>> hcache;     // key -> diag(H)
  S->hdiag.clear();
  const int pn = s + 1;                                          // patch nodes per axis
  const int np = dim == 2 ? pn : pn * pn;
  std::vector<double> Mp(np * np, 0.0), Lp(np * np, 0.0);
  if (dim == 2) {
    for (int e = 0; e < s; ++e)
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
          Mp[(e + x) * np + e + y] += M1[x][y];
          Lp[(e + x) * np + e + y] += L1[x][y];
        }
  } else {
    for (int e1 = 0; e1 < s; ++e1)
      for (int e2 = 0; e2 < s; ++e2)
        for (int a1 = 0; a1 < 2; ++a1)
          for (int a2 = 0; a2 < 2; ++a2)
            for (int b1 = 0; b1 < 2; ++b1)
              for (int b2 = 0; b2 < 2; ++b2) {
                const int r = (e1 + a1) * pn + e2 + a2, c = (e1 + b1) * pn + e2 + b2;
                Mp[r * np + c] += M1[a1][b1] * M1[a2][b2];
                Lp[r * np + c] += L1[a1][b1] * M1[a2][b2] + M1[a1][b1] * L1[a2][b2];
              }
  }
  int max_n = 0;
  for (auto& kv : faces) {
    const int na = std::get<0>(kv.first);
    int tax[2] = {0, 0}, ti = 0;
    for (int a = 0; a < dim; ++a)
      if (a != na) tax[ti++] = a;
    const int q0 = std::get<2>(kv.first), q1 = std::get<3>(kv.first);
    std::vector<int64_t> nodes = kv.second;
    std::sort(nodes.begin(), nodes.end());  // lexicographic in (i, j, k)
    for (int comp = 0; comp < dim; ++comp) {
      std::vector<int> pidx;
      std::vector<int64_t> dofs;
      for (int64_t n : nodes) {
        const int64_t d = dim * n + comp;
        if (S->fixed[d]) continue;
        const int c[3] = {(int)(n / (nn1 * nn2)), (int)((n / nn2) % nn1), (int)(n % nn2)};
        int pi = c[tax[0]] - q0 * s;
        if (dim == 3) pi = pi * pn + (c[tax[1]] - q1 * s);
        pidx.push_back(pi);
        dofs.push_back(d);
      }
      const int nb = (int)dofs.size();
      if (nb == 0) continue;
      max_n = std::max(max_n, nb);
      std::vector<double> Mf(nb * nb), Lf(nb * nb);
      for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
          Mf[a * nb + b] = Mp[pidx[a] * np + pidx[b]];
          Lf[a * nb + b] = Lp[pidx[a] * np + pidx[b]];
        }
      std::vector<double> key = Mf;
      key.insert(key.end(), Lf.begin(), Lf.end());
      key.push_back(nb);
      auto it = pcache.find(key);
      if (it == pcache.end()) {
        std::vector<double> mu, V;
        if (!gen_eig(nb, Lf, Mf, &mu, &V)) return "face mass matrix not positive definite";
        const bool singular = mu[0] <= 1e-12 * std::max(mu[nb - 1], 1.0);
        if (singular) S->n_singular_faces++;
        std::vector<double> lam(nb);
        // Eigenvalues at rounding level of a singular face are exactly zero (the
        // constants span the kernel of L_f); the fractional power would
        // otherwise amplify their rounding noise.
        const double zero_tol = 1e-12 * std::max(mu[nb - 1], 1.0);
        for (int a = 0; a < nb; ++a)
          lam[a] = singular ? 1.0 + (mu[a] <= zero_tol ? 0.0 : std::pow(mu[a], 1.0 - theta))
                            : std::pow(mu[a], 1.0 - theta);
        const int poff = (int)S->ptab.size();
        S->ptab.resize(poff + nb * nb);
        for (int a = 0; a < nb; ++a)
          for (int b = 0; b < nb; ++b) {
            double v = 0.0;
            for (int m = 0; m < nb; ++m) v += V[a * nb + m] * V[b * nb + m] / lam[m];
            S->ptab[poff + a * nb + b] = v;
          }
        // mean diag of H = M V diag(lam) V^T M
        std::vector<double> MV(nb * nb, 0.0);
        for (int a = 0; a < nb; ++a)
          for (int m = 0; m < nb; ++m) {
            double v = 0.0;
            for (int b = 0; b < nb; ++b) v += Mf[a * nb + b] * V[b * nb + m];
            MV[a * nb + m] = v;
          }
        double hsum = 0.0;
        std::vector<double> hd(nb, 0.0);
        for (int a = 0; a < nb; ++a) {
          for (int m = 0; m < nb; ++m) hd[a] += MV[a * nb + m] * MV[a * nb + m] * lam[m];
          hsum += hd[a];
        }
        hcache.emplace(key, hd);
        it = pcache.emplace(key, std::make_pair(poff, hsum / nb)).first;
      }
      const std::vector<double>& hd = hcache[key];
      S->hdiag.insert(S->hdiag.end(), hd.begin(), hd.end());
      S->blk_off.push_back((int)S->gamma_dof.size());
      S->blk_n.push_back(nb);
      S->blk_poff.push_back(it->second.first);
      S->blk_hmean.push_back(it->second.second);
      for (int64_t d : dofs) S->gamma_dof.push_back(d);
    }
  }
  S->max_blk_n = max_n;
  S->n_face_dofs = (int)S->gamma_dof.size();
  std::sort(cross_dofs.begin(), cross_dofs.end());
  for (int64_t d : cross_dofs) S->gamma_dof.push_back(d);
  S->dof_gamma.assign(S->n_dof, -1);
  for (size_t g = 0; g < S->gamma_dof.size(); ++g) S->dof_gamma[S->gamma_dof[g]] = (int32_t)g;

  // ---- subdomains: interior boxes, rings -----------------------------------
  S->subs.assign(S->n_sub, SubInfo{});
  S->ring_gidx.clear();
  S->ring_loc.clear();
  int maxbsz = 1, nbmax = 0;
  for (int qx = 0; qx < S->nsa[0]; ++qx)
    for (int qy = 0; qy < S->nsa[1]; ++qy)
      for (int qz = 0; qz < S->nsa[2]; ++qz) {
        const int id = (qx * S->nsa[1] + qy) * S->nsa[2] + qz;
        SubInfo& si = S->subs[id];
        const int q[3] = {qx, qy, qz};
        int hi[3];
        for (int a = 0; a < 3; ++a) {
          if (a >= dim) {
            si.lo[a] = 0;
            si.ilo[a] = 0;
            hi[a] = 0;
            continue;
          }
          si.lo[a] = q[a] * s;
          si.ilo[a] = q[a] == 0 ? 0 : q[a] * s + 1;
          hi[a] = q[a] == S->nsa[a] - 1 ? S->ne[a] : (q[a] + 1) * s - 1;
        }
        auto plane_all_fixed = [&](int x) {
          for (int j = si.ilo[1]; j <= hi[1]; ++j)
            for (int k = si.ilo[2]; k <= hi[2]; ++k)
              for (int comp = 0; comp < dim; ++comp)
                if (!S->fixed[dim * node_of(x, j, k) + comp]) return false;
          return true;
        };
        while (si.ilo[0] <= hi[0] && plane_all_fixed(si.ilo[0])) si.ilo[0]++;
        while (hi[0] >= si.ilo[0] && plane_all_fixed(hi[0])) hi[0]--;
        for (int a = 0; a < 3; ++a) si.icnt[a] = std::max(0, hi[a] - si.ilo[a] + 1);
        si.nb = si.icnt[0];
        si.bsz = dim * si.icnt[1] * (dim == 3 ? si.icnt[2] : 1);
        maxbsz = std::max(maxbsz, si.bsz);
        nbmax = std::max(nbmax, si.nb);
        si.ring_off = (int32_t)S->ring_gidx.size();
        const int pz = dim == 3 ? s + 1 : 1;
        for (int a = 0; a <= s; ++a)
          for (int b = 0; b <= s; ++b)
            for (int c = 0; c < pz; ++c) {
              const int64_t n = node_of(si.lo[0] + a, si.lo[1] + b, si.lo[2] + c);
              const int loc = (a * (s + 1) + b) * pz + c;
              for (int comp = 0; comp < dim; ++comp) {
                const int32_t g = S->dof_gamma[dim * n + comp];
                if (g < 0) continue;
                S->ring_gidx.push_back(g);
                S->ring_loc.push_back(loc * dim + comp);
              }
            }
        si.n_ring = (int32_t)S->ring_gidx.size() - si.ring_off;
      }
  S->BP = ((maxbsz + 31) / 32) * 32;
  S->nb_max = nbmax;
  const int64_t PC = (int64_t)S->BP * S->BP, PD = (int64_t)S->BP * (S->BP + 1) / 2;
  int64_t off = 0;
  for (auto& si : S->subs) {
    si.factor_off = off;
    off += (int64_t)si.nb * (PC + PD);
  }
  S->factor_elems = off;
  // owners of every Gamma DOF, in subdomain order
  const int64_t ng = (int64_t)S->gamma_dof.size();
  std::vector<int32_t> count(ng + 1, 0);
  for (int32_t g : S->ring_gidx) count[g + 1]++;
  S->owner_ptr.assign(ng + 1, 0);
  for (int64_t g = 0; g < ng; ++g) S->owner_ptr[g + 1] = S->owner_ptr[g] + count[g + 1];
  S->owner_idx.assign(S->ring_gidx.size(), 0);
  std::vector<int32_t> fill(S->owner_ptr.begin(), S->owner_ptr.end() - 1);
  for (size_t r = 0; r < S->ring_gidx.size(); ++r) S->owner_idx[fill[S->ring_gidx[r]]++] = (int32_t)r;
  // the same owners as a fixed-width table (one vector load per Gamma DOF)
  S->max_owners = dim == 2 ? 4 : 8;
  S->owner_pad.assign((size_t)ng * S->max_owners, -1);
  for (int64_t g = 0; g < ng; ++g) {
    if (S->owner_ptr[g + 1] - S->owner_ptr[g] > S->max_owners) return "internal: too many owners";
    for (int o = S->owner_ptr[g]; o < S->owner_ptr[g + 1]; ++o)
      S->owner_pad[(size_t)g * S->max_owners + (o - S->owner_ptr[g])] = S->owner_idx[o];
  }
  // owner-major destination of every ring slot: subdomain contributions land
  // in the max_owners consecutive entries of their Gamma DOF (unused ones stay 0)
  S->ring_dst.assign(S->ring_gidx.size(), -1);
  for (int64_t g = 0; g < ng; ++g)
    for (int k = 0; k < S->max_owners; ++k) {
      const int32_t slot = S->owner_pad[(size_t)g * S->max_owners + k];
      if (slot >= 0) S->ring_dst[slot] = (int32_t)(g * S->max_owners + k);
    }
  return "";
}

void interface_operator(const Setup& S, int comp, std::vector<int32_t>* pos, std::vector<int64_t>* rowptr,
                        std::vector<int32_t>* col, std::vector<double>* M, std::vector<double>* L) {
  const int dim = S.dim, s = S.sub;
  // Gamma positions of this component, and the local row of each node
  std::vector<int32_t> local(S.n_nodes, -1);
  pos->clear();
  for (size_t k = 0; k < S.gamma_dof.size(); ++k) {
    const int64_t d = S.gamma_dof[k];
    if (d % dim != comp) continue;
    local[d / dim] = (int32_t)pos->size();
    pos->push_back((int32_t)k);
  }
  const size_t n = pos->size();
  std::vector<std::map<int32_t, std::pair<double, double>>> rows(n);
  auto node = [&](const int c[3]) -> int64_t {
    return ((int64_t)c[0] * S.nn[1] + c[1]) * S.nn[2] + c[2];
  };
  auto add = [&](const int64_t* nodes, int m, const double* Me, const double* Le) {
    for (int a = 0; a < m; ++a) {
      const int32_t ra = local[nodes[a]];
      if (ra < 0) continue;
      for (int b = 0; b < m; ++b) {
        const int32_t rb = local[nodes[b]];
        if (rb < 0) continue;
        auto& e = rows[ra][rb];
        e.first += Me[a * m + b];
        e.second += Le[a * m + b];
      }
    }
  };
  const double M1[4] = {2.0 / 6, 1.0 / 6, 1.0 / 6, 2.0 / 6};
  const double L1[4] = {1.0, -1.0, -1.0, 1.0};
  if (dim == 2) {
    for (int a = 0; a < 2; ++a) {  // edges along axis a on the interface lines of the other axis
      const int b = 1 - a;
      for (int y = s; y < S.ne[b]; y += s)
        for (int x = 0; x < S.ne[a]; ++x) {
          int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
          c0[a] = x;
          c1[a] = x + 1;
          c0[b] = c1[b] = y;
          const int64_t nodes[2] = {node(c0), node(c1)};
          add(nodes, 2, M1, L1);
        }
    }
  } else {
    // unit-square Q1: M = M1 (x) M1, L = L1 (x) M1 + M1 (x) L1, nodes (i, j) -> 2 i + j
    double M2[16], L2[16];
    for (int i1 = 0; i1 < 2; ++i1)
      for (int j1 = 0; j1 < 2; ++j1)
        for (int i2 = 0; i2 < 2; ++i2)
          for (int j2 = 0; j2 < 2; ++j2) {
            const int r = 2 * i1 + j1, c = 2 * i2 + j2;
            M2[r * 4 + c] = M1[i1 * 2 + i2] * M1[j1 * 2 + j2];
            L2[r * 4 + c] = L1[i1 * 2 + i2] * M1[j1 * 2 + j2] + M1[i1 * 2 + i2] * L1[j1 * 2 + j2];
          }
    for (int a = 0; a < 3; ++a) {  // quads normal to axis a on the interface planes
      const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
      for (int x = s; x < S.ne[a]; x += s)
        for (int eb = 0; eb < S.ne[b]; ++eb)
          for (int ec = 0; ec < S.ne[c]; ++ec) {
            int64_t nodes[4];
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j) {
                int q[3];
                q[a] = x;
                q[b] = eb + i;
                q[c] = ec + j;
                nodes[2 * i + j] = node(q);
              }
            add(nodes, 4, M2, L2);
          }
    }
  }
  rowptr->assign(n + 1, 0);
  col->clear();
  M->clear();
  L->clear();
  for (size_t r = 0; r < n; ++r) {
    for (const auto& kv : rows[r]) {
      col->push_back(kv.first);
      M->push_back(kv.second.first);
      L->push_back(kv.second.second);
    }
    (*rowptr)[r + 1] = (int64_t)col->size();
  }
}


// ---- global interface preconditioner (Sec. 3-4): host set-up ---------------
namespace {

// Inverse of the SPD n x n matrix A (row-major) by Cholesky; false if a pivot
// is not positive.
bool spd_inverse(int n, const std::vector<double>& A, std::vector<double>* inv) {
  std::vector<double> Lc(A);
  for (int j = 0; j < n; ++j) {
    double d = Lc[j * n + j];
    for (int k = 0; k < j; ++k) d -= Lc[j * n + k] * Lc[j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    Lc[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = Lc[i * n + j];
      for (int k = 0; k < j; ++k) v -= Lc[i * n + k] * Lc[j * n + k];
      Lc[i * n + j] = v / d;
    }
  }
  inv->assign((size_t)n * n, 0.0);
  std::vector<double> e(n), y(n);
  for (int c = 0; c < n; ++c) {
    // L y = e_c, L^T x = y
    for (int i = 0; i < n; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= Lc[i * n + k] * y[k];
      y[i] = v / Lc[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < n; ++k) v -= Lc[k * n + i] * e[k];
      e[i] = v / Lc[i * n + i];
    }
    for (int i = 0; i < n; ++i) (*inv)[(size_t)i * n + c] = e[i];
  }
  return true;
}

}  // namespace

std::string build_global_prec(const Setup& S, int comp, GPHost* G) {
  interface_operator(S, comp, &G->pos, &G->rowptr, &G->col, &G->M, &G->L);
  const int n = (int)G->pos.size();
  G->Mdiag.assign(n, 0.0);
  G->Ldiag.assign(n, 0.0);
  G->Minv_diag.assign(n, 0.0);
  G->cross_inv.assign(n, 0.0);
  std::vector<char> anchored(n, 0);
  for (int i = 0; i < n; ++i) {
    double rs = 0.0, amax = 0.0;
    for (int64_t q = G->rowptr[i]; q < G->rowptr[i + 1]; ++q) {
      if (G->col[q] == i) {
        G->Mdiag[i] = G->M[q];
        G->Ldiag[i] = G->L[q];
      }
      rs += G->L[q];
      amax = std::max(amax, std::fabs(G->L[q]));
    }
    if (!(G->Mdiag[i] > 0.0) || !(G->Ldiag[i] > 0.0)) return "interface operator with an empty row";
    G->Minv_diag[i] = 1.0 / G->Mdiag[i];
    G->cross_inv[i] = 1.0 / G->Ldiag[i];
    // a row whose Laplacian entries do not sum to zero touches a removed
    // (clamped) node: it anchors its connected part of the interface
    anchored[i] = std::fabs(rs) > 1e-12 * amax;
  }
  // singular L: a connected part of the interface graph without an anchor
  std::vector<int> part(n, -1), stack;
  G->singular = false;
  for (int s0 = 0; s0 < n && !G->singular; ++s0) {
    if (part[s0] >= 0) continue;
    bool anch = false;
    stack.assign(1, s0);
    part[s0] = s0;
    while (!stack.empty()) {
      const int i = stack.back();
      stack.pop_back();
      anch = anch || anchored[i];
      for (int64_t q = G->rowptr[i]; q < G->rowptr[i + 1]; ++q) {
        const int j = G->col[q];
        if (part[j] < 0) {
          part[j] = s0;
          stack.push_back(j);
        }
      }
    }
    if (!anch) G->singular = true;
  }
  // faces: the face-local preconditioner's blocks of this component, as
  // contiguous ranges of local rows (Gamma positions are ascending in pos)
  std::vector<int32_t> local(S.gamma_dof.size(), -1);
  for (int i = 0; i < n; ++i) local[G->pos[i]] = i;
  G->row_face.assign(n, -1);
  G->face_l0.clear();
  G->face_n.clear();
  G->face_inv_off.clear();
  G->face_inv.clear();
  for (size_t b = 0; b < S.blk_off.size(); ++b) {
    const int off = S.blk_off[b], nb = S.blk_n[b];
    if (nb <= 0 || S.gamma_dof[off] % S.dim != comp) continue;
    const int l0 = local[off];
    if (l0 < 0) return "face block outside its component";
    for (int a = 0; a < nb; ++a)
      if (local[off + a] != l0 + a) return "face block not contiguous in its component";
    std::vector<double> A((size_t)nb * nb, 0.0), inv;
    for (int a = 0; a < nb; ++a)
      for (int64_t q = G->rowptr[l0 + a]; q < G->rowptr[l0 + a + 1]; ++q) {
        const int cb = G->col[q] - l0;
        if (cb >= 0 && cb < nb) A[(size_t)a * nb + cb] = G->L[q];
      }
    if (!spd_inverse(nb, A, &inv)) return "face Laplacian not positive definite";
    const int f = (int)G->face_l0.size();
    G->face_l0.push_back(l0);
    G->face_n.push_back(nb);
    G->face_inv_off.push_back((int64_t)G->face_inv.size());
    G->face_inv.insert(G->face_inv.end(), inv.begin(), inv.end());
    for (int a = 0; a < nb; ++a) G->row_face[l0 + a] = f;
  }
  return "";
}

}  // namespace ddel
