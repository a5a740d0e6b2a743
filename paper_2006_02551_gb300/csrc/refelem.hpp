// Reference-tetrahedron operators for nodal DG of order N, built in FP64 on
// the host (Section II.A: reference matrices M, S, F of eqs. 14, 16, 17;
// V_q, P_q of eqs. 20, 21).
#pragma once
#include <vector>

namespace wadg {

int n_nodes(int N);
int n_face_nodes(int N);

struct RefOps {
  int N = 0, Np = 0, Nfp = 0, Nq = 0;
  std::vector<double> r, s, t;        // nodes [Np]
  std::vector<int> bary;              // integer barycentrics [Np][4] (sum N)
  std::vector<double> V, Vinv, Minv;  // [Np][Np] row-major
  std::vector<double> Dr, Ds, Dt;     // [Np][Np]
  std::vector<int> Fmask;             // [4][Nfp] volume node of face node
  std::vector<double> LIFT;           // [Np][4 Nfp]
  // volume quadrature [Nq]: the rule's Nq_rule points, then zero-weight
  // padding points (at the centroid) up to the kernels' capacity Nq
  int Nq_rule = 0;
  std::vector<double> rq, sq, tq, wq;
  std::vector<double> Vq;             // [Nq][Np]
  std::vector<double> Pq;             // [Np][Nq]
  // face-node permutation table: for local face f, neighbour face nf and
  // vertex rotation rot (code = nf*6 + rot), the neighbour's volume node
  // that coincides with face node m of face f: [4][24][Nfp]
  std::vector<int> fperm;
  // the same table as face-node indices of the neighbour's face: [4][24][Nfp]
  std::vector<int> fmap;
  std::vector<double> lagrange_at(double r, double s, double t) const;  // [Np]
};

// Stroud conical-product rule on the reference tetrahedron with n points per
// collapsed direction (n^3 points, exact for polynomials of degree 2n - 1).
void stroud_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& t,
                 std::vector<double>& w);

// Builds all operators (with the default conical-product volume rule of
// degree 2N+1); returns false (and a message) on failure.
bool build_ref_ops(int N, RefOps& out, const char** err);

// Replaces the volume quadrature (eqs. 20, 21) by the rule (r, s, t, w),
// padded with zero-weight points up to pad_to points, and rebuilds V_q and
// P_q = M^-1 V_q^T W.  Refuses (false and a message) a rule with a weight
// that is not positive, a point outside the tetrahedron, or one that does not
// integrate degree 2N exactly (P_q V_q must be the identity to 1e-10).
bool set_volume_rule(RefOps& o, const std::vector<double>& r, const std::vector<double>& s,
                     const std::vector<double>& t, const std::vector<double>& w, int pad_to,
                     const char** err);

// the six permutations of three face vertices used to encode rotations
extern const int kFacePerm[6][3];
// local vertex triples of the four faces (t=-1, s=-1, r+s+t=-1, r=-1)
extern const int kFaceVerts[4][3];

}  // namespace wadg
