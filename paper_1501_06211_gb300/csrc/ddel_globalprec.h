// Global interface preconditioner (inverse Lanczos, Sec. 3) and the vector
// kernels of the full-system flexible GMRES: device layout and launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ddel_internal.h"

namespace ddel {

constexpr int kLz = 32;  // most inverse Lanczos steps (DDEL_MAX_LANCZOS)

// One displacement component of the interface: its rows are the component's
// free Gamma DOFs in Gamma order (pos), M and L the assembled interface mass
// and Laplacian (CSR), and the inner preconditioner of the solves with L:
// dense inverses of L on each face (rows face_l0 .. face_l0 + face_n - 1;
// row_face[i] = the face of row i, -1 at cross points, where 1 / L_ii is used).
struct GPComp {
  int n = 0;
  const int32_t* pos = nullptr;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* M = nullptr;
  const double* L = nullptr;
  const double* Mdiag = nullptr;
  const double* Ldiag = nullptr;
  const double* Minv_diag = nullptr;
  const double* cross_inv = nullptr;  // 1 / L_ii (every row; used at cross points)
  const int32_t* row_face = nullptr;
  const int32_t* face_l0 = nullptr;
  const int32_t* face_n = nullptr;
  const int64_t* face_inv_off = nullptr;
  const double* face_inv = nullptr;
  double* w = nullptr;     // scaling W_ii of the last application
  double* work = nullptr;  // global_prec_work_elems(n, k) doubles
};

struct GPDev {
  GPComp c[3];
  int ncomp = 0;
};

// Host form of one component (built from a Setup).
struct GPHost {
  std::vector<int32_t> pos;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> M, L, Mdiag, Ldiag, Minv_diag, cross_inv;
  std::vector<int32_t> row_face, face_l0, face_n;
  std::vector<int64_t> face_inv_off;
  std::vector<double> face_inv;
  bool singular = false;  // a connected part of the interface meets no clamped node
};

// Builds component comp of the global preconditioner from the set-up: the
// interface operators of interface_operator, the face groups of the
// face-local preconditioner (its blocks of this component) and their dense
// inverses of L, and the singularity test of L.  Returns an error message or
// an empty string.
std::string build_global_prec(const Setup& S, int comp, GPHost* out);

size_t global_prec_work_elems(int n, int ksteps);
cudaError_t launch_global_prec(const GPDev& gd, const double* r, double* z, const double* diagG, double theta,
                               int ksteps, double inner_tol, double mass_tol, int scaling, double* out,
                               cudaStream_t st);
// h[j] (+)= V_j . w for j < nv (V_j = V + j ld), deterministic; partial: multi_dot_partials(nv) doubles.
void launch_multi_dot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* partial,
                      double* h, int accumulate, cudaStream_t st);
size_t multi_dot_partials(int nv);
// w -= sum_j h[j] V_j, or (overwrite) w = sum_j h[j] V_j.
void launch_multi_axpy(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n, int overwrite,
                       cudaStream_t st);
// out = in / h[idx] (device scalar), or out = in / s0 when idx < 0.
void launch_scale_gm(const double* in, double* out, int64_t n, const double* h, int idx, double s0,
                     cudaStream_t st);
// out[g] = in[gamma_dof[g]]
void launch_gather_gamma(const int64_t* gd, int64_t ng, const double* in, double* out, cudaStream_t st);

}  // namespace ddel
