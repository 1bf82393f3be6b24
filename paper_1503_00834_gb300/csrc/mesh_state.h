// The mesh handle behind chorus_mesh and the internal calls that the batched-shell layer
// (batch.cu) makes on it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "chorus.h"
#include "internal.h"
#include "mesh_builder.h"
#include "sd_tables.h"

struct chorus_mesh_s {
  int p = 0, N = 0;
  int64_t E = 0;
  double r_inner = 0, r_outer = 0;
  chorus::HostMesh host;
  chorus::Tables1D tab;
  chorus::LaunchSet L{};
  int tile = 0;  // FP32 tile shape in use (index into the order's built tile shapes)
  chorus::OpsArg<double> ops64{};
  chorus::OpsArg<float> ops32{};
  // device mesh arrays
  int* d_nbr = nullptr;
  int* d_code = nullptr;
  double* d_Sf64 = nullptr;
  double* d_invJ64 = nullptr;
  double* d_x64 = nullptr;
  double* d_wJ = nullptr;  // w_i w_j w_k |J| at the solution points (reductions)
  float* d_Sf32 = nullptr;
  float* d_invJ32 = nullptr;
  float* d_x32 = nullptr;
  unsigned* d_err = nullptr;
  // face list (element, local face): the interior faces from their lower element, then the wall faces
  int2* d_faces = nullptr;
  int n_ifaces = 0, n_wfaces = 0;
  // prepared background
  bool prepared = false;
  chorus_params prep{};
  double* d_Q0 = nullptr;     // [E][5][N3] FP64 polytrope at rest
  float* d_bg = nullptr;      // [E][2][N3]
  float* d_grho0 = nullptr;   // [E][3][N3]
  float* d_bgT = nullptr;     // [E][6][2][N2]
  float* d_R0 = nullptr;      // [E][5][N3]
  double* d_red = nullptr;    // reduction partials
  // measurement: event pairs around launches while timing is enabled
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  // attached learned closure (p = 2 meshes): record pointer and its per-stage output buffer
  // radial radiative-diffusivity profile at the flux points (active when the params vary it)
  bool kr_active = false;
  double kr_coef[3] = {0, 0, 0};
  double* d_kr64 = nullptr;
  float* d_kr32 = nullptr;
  // well-balanced perturbation residual: R(Q0) is left out, so the discrete background is steady
  bool well_balanced = false;
  const void* closure = nullptr;
  void* closure_buf = nullptr;
  // chorus_rk_step_host: the copy stream and the events of its element chunks (in and out)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[18] = {};
};

namespace chorus {

// Seeded perturbation (as chorus_state_init, FP32 form) of elements [e0, e0 + ne) of a prepared
// mesh, indexing the points from the range's first point, so that the range gets the state a
// standalone mesh of those elements gets.
chorus_status mesh_init_range(chorus_mesh_s* m, uint64_t seed, double amp, float* Q, int64_t e0, int64_t ne,
                              cudaStream_t st);

// chorus_reduce (FP32 form) over elements [e0, e0 + ne).  Synchronises.
chorus_status mesh_reduce_range(chorus_mesh_s* m, const float* Q, int64_t e0, int64_t ne, double out[4],
                                cudaStream_t st);

// Select the FP32 tile shape `tile` (0 <= tile < n_tiles(p)); returns the elements per CTA or -1.
int mesh_set_tile(chorus_mesh_s* m, int tile);

// One stage of an explicit SSP scheme: residual of `src`, fused combination into `dst` (and
// optionally a second output), traces of `dst` for the next stage.
struct Stage {
  int src, dst;           // buffer ids: 0 u (the caller's state), 1 s, 2 A, 3 B
  int un;                 // first extra input
  double a, b, c;         // dst = a un + b src + c dt L(src)
  int un2, out2;          // -1: none
  double a2, b2, c2;      // out2 = a2 un2 + b2 src + c2 dt L(src)
};
// Stage lists: scheme 0 SSP-RK3, 1 SSP-RK(5,4).
const std::vector<Stage>& stages_of(int scheme);

// The device arrays and constants of an FP32 RK stage of a prepared mesh, for the caller's state u
// and workspace ws (the persistent batch step builds its kernel arguments from them).
struct StagePtrs {
  MeshArg<float> m;
  OpsArg<float> ops;
  PhysArg<float> ph;
  BgArg bg;
  float* buf[4];  // stage buffers: u, s, A, B (ids of Stage)
  float *Ta, *Tb, *Tv, *G, *Fc;
  const int2* faces;
  int nf, nw;
  unsigned* err;
};
chorus_status mesh_stage_ptrs(chorus_mesh_s* m, const chorus_params& P, float* u, void* ws, StagePtrs* out);

// Persistent batch step (batch_persist.cu): one SSP-RK3 step of up to four order groups (slot
// p - 2, null where the order is absent) as three cooperative launches, one per stage, each running
// the stage's phases for every order with bounded grid barriers between them.  sync: 5 device words
// of scratch.  CHORUS_EUNSUPPORTED when the device cannot launch it or a group has a radial kappa_r.
chorus_status persist_rk3_step(StagePtrs* const groups[4], double dt, unsigned* sync, cudaStream_t st);
// CTAs of the persistent launch (all resident at once), 0 when unavailable.
int persist_grid();

}  // namespace chorus
