// Host mesh builder: face pairing and orientation, wall tagging, 20-node geometry and metrics
// (paper Section 3 Eqs. 10-12, Section 5), all in double precision.
#pragma once
#include <stdint.h>

#include <vector>

#include "sd_tables.h"

namespace chorus {

struct HostMesh {
  int p = 0, N = 0;
  int64_t E = 0;
  std::vector<int> nbr;      // [E][6] neighbour element, -1 inner wall, -2 outer wall
  std::vector<int> code;     // [E][6] neighbour face * 8 + orientation bits (swap, flip1, flip2)
  std::vector<double> Sf;    // [E][3][3][N+1][N2]
  std::vector<double> x;     // [E][3][N3]
  std::vector<double> detJ;  // [E][N3]
  double h_min = 0.0, volume = 0.0;
  int64_t n_interior_faces = 0, n_wall_faces = 0;
};

// Returns 0 on success, 1 for invalid arguments, 4 for an invalid mesh (chorus_status codes).
int build_mesh(int64_t n_nodes, const double* node_xyz, int64_t n_elem, const int64_t* hex20, int p,
               double r_inner, double r_outer, int metric_mode, const Tables1D& tab, HostMesh* out,
               const char** why);

}  // namespace chorus
