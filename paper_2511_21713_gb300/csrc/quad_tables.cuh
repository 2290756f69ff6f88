// Quadrature tables of the device code.
//
// Tetrahedra: the symmetric 14-point rule exact for degree-5 polynomials
// (orbits S31(a1), S31(a2), S22(c); weights normalised to sum 1).
// Triangles: the symmetric 6-point rule exact for degree 4 (Dunavant 1985,
// orbits S21(b1), S21(b2); weights normalised to sum 1).
// Both are the "fourth-order Gaussian quadrature" of the paper's Sec. 3
// fixed to concrete published rules.
#pragma once

namespace pbfb {

#define PBFB_T_A1 0.09273525031089122640
#define PBFB_T_A2 0.31088591926330060980
#define PBFB_T_C3 0.04550370412564964949
#define PBFB_T_W1 0.07349304311636194954
#define PBFB_T_W2 0.11268792571801585080
#define PBFB_T_W3 0.04254602077708146644
#define PBFB_T_B1 (1.0 - 3.0 * PBFB_T_A1)
#define PBFB_T_B2 (1.0 - 3.0 * PBFB_T_A2)
#define PBFB_T_D3 (0.5 - PBFB_T_C3)

// barycentric coordinates (l0, l1, l2, l3) of the 14 tet points
static __constant__ double c_tet_l[14][4] = {
    {PBFB_T_B1, PBFB_T_A1, PBFB_T_A1, PBFB_T_A1}, {PBFB_T_A1, PBFB_T_B1, PBFB_T_A1, PBFB_T_A1},
    {PBFB_T_A1, PBFB_T_A1, PBFB_T_B1, PBFB_T_A1}, {PBFB_T_A1, PBFB_T_A1, PBFB_T_A1, PBFB_T_B1},
    {PBFB_T_B2, PBFB_T_A2, PBFB_T_A2, PBFB_T_A2}, {PBFB_T_A2, PBFB_T_B2, PBFB_T_A2, PBFB_T_A2},
    {PBFB_T_A2, PBFB_T_A2, PBFB_T_B2, PBFB_T_A2}, {PBFB_T_A2, PBFB_T_A2, PBFB_T_A2, PBFB_T_B2},
    {PBFB_T_D3, PBFB_T_D3, PBFB_T_C3, PBFB_T_C3}, {PBFB_T_D3, PBFB_T_C3, PBFB_T_D3, PBFB_T_C3},
    {PBFB_T_D3, PBFB_T_C3, PBFB_T_C3, PBFB_T_D3}, {PBFB_T_C3, PBFB_T_D3, PBFB_T_D3, PBFB_T_C3},
    {PBFB_T_C3, PBFB_T_D3, PBFB_T_C3, PBFB_T_D3}, {PBFB_T_C3, PBFB_T_C3, PBFB_T_D3, PBFB_T_D3}};
static __constant__ double c_tet_w[14] = {PBFB_T_W1, PBFB_T_W1, PBFB_T_W1, PBFB_T_W1,
                                          PBFB_T_W2, PBFB_T_W2, PBFB_T_W2, PBFB_T_W2,
                                          PBFB_T_W3, PBFB_T_W3, PBFB_T_W3,
                                          PBFB_T_W3, PBFB_T_W3, PBFB_T_W3};

#define PBFB_S_B1 0.44594849091596488632
#define PBFB_S_B2 0.09157621350977074346
#define PBFB_S_W1 0.22338158967801146570
#define PBFB_S_W2 0.10995174365532186764

// barycentric coordinates of the 6 triangle points and their weights
static __constant__ double c_tri_b[6][3] = {
    {1.0 - 2.0 * PBFB_S_B1, PBFB_S_B1, PBFB_S_B1}, {PBFB_S_B1, 1.0 - 2.0 * PBFB_S_B1, PBFB_S_B1},
    {PBFB_S_B1, PBFB_S_B1, 1.0 - 2.0 * PBFB_S_B1}, {1.0 - 2.0 * PBFB_S_B2, PBFB_S_B2, PBFB_S_B2},
    {PBFB_S_B2, 1.0 - 2.0 * PBFB_S_B2, PBFB_S_B2}, {PBFB_S_B2, PBFB_S_B2, 1.0 - 2.0 * PBFB_S_B2}};
static __constant__ double c_tri_w[6] = {PBFB_S_W1, PBFB_S_W1, PBFB_S_W1,
                                         PBFB_S_W2, PBFB_S_W2, PBFB_S_W2};

// host copies (same values) for host-side setup
static const double h_tri_b[6][3] = {
    {1.0 - 2.0 * PBFB_S_B1, PBFB_S_B1, PBFB_S_B1}, {PBFB_S_B1, 1.0 - 2.0 * PBFB_S_B1, PBFB_S_B1},
    {PBFB_S_B1, PBFB_S_B1, 1.0 - 2.0 * PBFB_S_B1}, {1.0 - 2.0 * PBFB_S_B2, PBFB_S_B2, PBFB_S_B2},
    {PBFB_S_B2, 1.0 - 2.0 * PBFB_S_B2, PBFB_S_B2}, {PBFB_S_B2, PBFB_S_B2, 1.0 - 2.0 * PBFB_S_B2}};
static const double h_tri_w[6] = {PBFB_S_W1, PBFB_S_W1, PBFB_S_W1,
                                  PBFB_S_W2, PBFB_S_W2, PBFB_S_W2};

// index of the unordered local pair (a, b) of a tet in the 10-entry symmetric storage
__host__ __device__ inline int sym10(int a, int b) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  // rows: (0,0..3) -> 0..3, (1,1..3) -> 4..6, (2,2..3) -> 7..8, (3,3) -> 9
  return lo == 0 ? hi : (lo == 1 ? 3 + hi : (lo == 2 ? 5 + hi : 9));
}

}  // namespace pbfb
