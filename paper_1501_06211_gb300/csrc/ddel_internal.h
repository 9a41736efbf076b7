// Internal data layout shared by the host set-up (C++) and the CUDA kernels.
// Plain structs only: the set-up fills them on the host and copies them to
// device memory once per context.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace ddel {

constexpr int kMaxDim = 3;

// Error words written by kernels (the host reads them after a phase).
enum : int { kErrNone = 0, kErrPivot = 1, kErrTimeout = 2, kErrBadRho = 3 };

// One subdomain Omega_i (Sec. 1).  Its closure covers nodes lo[a] .. lo[a]+sub
// on every axis.  Its interior DOFs (the set I_i of eq. NumberFive) are the
// free DOFs of the node box ilo[a] .. ilo[a]+icnt[a]-1; they are ordered plane
// by plane along axis 0, which makes K_{I_i I_i} block tridiagonal with nb
// blocks of bsz rows each (padded to the context's block size BP).
struct SubInfo {
  int32_t lo[kMaxDim];
  int32_t ilo[kMaxDim];
  int32_t icnt[kMaxDim];
  int32_t nb;         // number of interior planes (blocks)
  int32_t bsz;        // DOF rows per block = dim * prod(icnt[1..])
  int32_t ring_off;   // first entry of this subdomain in the ring tables
  int32_t n_ring;     // number of free Gamma DOFs in the closure
  int64_t factor_off; // element offset of this subdomain's factor
};

// Host-side result of the set-up (all sizes and tables).
struct Setup {
  int dim = 2;
  int ne[kMaxDim] = {0, 0, 1};  // elements per axis
  int nn[kMaxDim] = {1, 1, 1};  // nodes per axis
  int sub = 1;
  int nsa[kMaxDim] = {1, 1, 1};  // subdomains per axis
  int n_sub = 0;
  int64_t n_nodes = 0, n_dof = 0, n_elem = 0;
  std::vector<uint8_t> fixed;     // n_dof
  std::vector<double> f;          // n_dof (loads of the BC description)
  std::vector<double> Ke;         // (dim*2^dim)^2, unit E, row-major
  // Gamma
  std::vector<int64_t> gamma_dof; // n_gamma
  std::vector<int32_t> dof_gamma; // n_dof -> gamma index or -1
  // subdomains
  std::vector<SubInfo> subs;
  int BP = 32;                    // padded block size (multiple of 32)
  int nb_max = 0;
  int64_t factor_elems = 0;       // per precision, in elements
  std::vector<int32_t> ring_gidx; // gamma index per ring slot
  std::vector<int32_t> ring_loc;  // local closure DOF (node*dim + comp)
  std::vector<int32_t> owner_ptr; // n_gamma + 1
  std::vector<int32_t> owner_idx; // ring slots contributing to each gamma DOF
  int max_owners = 4;             // 2^(dim-1) ... 2^dim: 4 in 2D, 8 in 3D
  std::vector<int32_t> owner_pad; // n_gamma * max_owners ring slots, -1 padded
  std::vector<int32_t> ring_dst;  // per ring slot: g * max_owners + (rank among g's owners)
  // preconditioner (face blocks first, then cross DOFs)
  int n_face_dofs = 0;
  std::vector<int32_t> blk_off, blk_n, blk_poff;  // per (face, component) block
  std::vector<double> blk_hmean;                  // mean of diag(H) per block
  std::vector<double> hdiag;                      // diag(H_f) per face DOF
  std::vector<double> ptab;                       // concatenated dense H^-1 (row-major)
  int max_blk_n = 0;
  int n_singular_faces = 0;
};

// Builds everything above.  Returns an empty string on success, else an error
// message (invalid sizes, material, or boundary description).
std::string build_setup(int dim, const int ne[3], int sub, double E, double nu, int plane_stress,
                        uint32_t clamp_faces, const uint8_t* fixed_dof, int n_point,
                        const int64_t* point_node, const double* point_force, int traction_face,
                        const double traction[3], const double body_force[3], double theta, Setup* out);

// Element stiffness for unit E by 2-point Gauss quadrature (exact for Q1/H8
// on unit elements), local node order (0,0),(1,0),(1,1),(0,1) [then z=1].
void element_stiffness(int dim, double nu, int plane_stress, std::vector<double>* Ke);

// Mass and Laplacian of eq. NumberEight assembled on all of Gamma for one
// displacement component (the form of the paper's Tables 1-3): unit-edge P1
// (2D) / unit-square Q1 (3D) element matrices over the facets that lie on
// Gamma -- those whose normal coordinate is an interior multiple of the
// subdomain edge -- restricted to the component's free Gamma DOFs.  Rows and
// columns follow the Gamma order (pos: the Gamma positions of the rows);
// CSR with ascending columns.
void interface_operator(const Setup& S, int comp, std::vector<int32_t>* pos, std::vector<int64_t>* rowptr,
                        std::vector<int32_t>* col, std::vector<double>* M, std::vector<double>* L);

// Generalized symmetric eigenproblem L V = M V diag(mu), V^T M V = I, by a
// Cholesky reduction and cyclic Jacobi rotations.  n <= 128.  Returns false if
// M is not positive definite.
bool gen_eig(int n, const std::vector<double>& L, const std::vector<double>& M,
             std::vector<double>* mu, std::vector<double>* V);

}  // namespace ddel
