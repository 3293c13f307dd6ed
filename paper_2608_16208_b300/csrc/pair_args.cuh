// Arguments of the per-pair pipeline kernel (shared by kernel modes and assembly).
#pragma once
#include "bie_internal.cuh"

namespace bie {

struct PairArgs {
  SurfP S;
  GL16 gl;
  int Np, Mt, M, P, T, L;
  double h, k;
  int64_t N, n_pairs, p0;          // p0: first enumerated pair of this launch
  int enumerate;                 // 1: pair p enumerates every (node, delta, g, theta) of the surface
  const double* t_nodes;
  const double* pts;
  const double* ring_t;
  const double* ring_r;
  const double* ring_n;
  const cplx* tw;
  const int64_t* rows;
  const int32_t* srcs;
  double* modes_out;             // [p][Mt+1] complex, or null
  cplx* weights_out;             // [p][Mt] complex, or null
  int* status;
};

PairArgs make_pair_args(bie_surface s, double k);
bie_status launch_pairs(bie_surface s, const PairArgs& a);

}  // namespace bie
