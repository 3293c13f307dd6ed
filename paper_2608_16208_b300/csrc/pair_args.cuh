// Arguments of the per-pair pipeline kernel (shared by kernel modes and assembly).
#pragma once
#include "bie_internal.cuh"

namespace bie {

struct PairArgs {
  SurfP S;
  GL16 gl;
  int Np, Mt, M, P, T, L;         // P: Toeplitz transform length; L: highest A_m index
  int kernels;                    // BIE_KERNEL_S and at most one of BIE_KERNEL_K, BIE_KERNEL_KP
  int kprime;                     // the double layer of this launch is K' (tau_0 with the target's normal)
  int out_nk, out_k0;             // modes_out holds out_nk kernels per pair; this launch writes from slot out_k0
  double h, k;
  int64_t N, n_pairs, p0;         // p0: first enumerated pair of this launch
  int enumerate;                  // 1: pair p enumerates every (node, delta, g, theta) of the surface
  const double* t_nodes;
  const double* pts;
  const double* nrm;              // unit normals of the nodes (the target's normal of K')
  const double* ring_t;
  const double* ring_r;
  const double* ring_n;
  const cplx* tw;
  const float4* twf;              // twiddles as double words
  const double* thg;              // [Mt][3]: th_q, sin(th_q/2), cos(th_q/2)
  const double* rec;              // recurrence coefficient table, 4 doubles per m (see pair_modes.cu)
  int rec_len;
  double* scratch;                // per resident warp: pair_scratch_per_warp(L, K) doubles
  int64_t scratch_per_warp;       // doubles
  const int64_t* rows;
  const int32_t* srcs;
  double* modes_out;              // [p][nk][Mt+1] complex, or null
  cplx* weights_out;              // [kernel][p][Mt] complex (kernel-major when both), or null
  int64_t weights_stride;         // complex elements between the S and K weight blocks
  int64_t out_base, out_mod;      // output slot of pair p: (out_base + p) % out_mod when out_mod > 0
  int64_t w_ld;                   // complex elements between consecutive weight rows (Mt by default)
  int weights_dw;                 // single layer: weights as double words (re.h, re.l, im.h, im.l)
  int fp64_transforms;            // single layer, split launch: transforms in FP64 instead of double words
  int* status;
  // single layer, split launch: one record per pair of the chunk, written by the root kernel
  double* rec_hdr;                // [pair][8]: a, e^{-b}, 1 - e^{-b}, sin(a/2), cos(a/2), valid
  float4* rec_E;                  // [pair][33]: e^{i l a}, l < 32, and e^{32 i a} as double words
  double* rec_A;                  // [pair][L + 1]: A_m as double words
  double* rec_R2;                 // [pair][Mt]: rho^2 on the ring
};

// Per-warp scratch (doubles): A_m (and D_m with the double layer) as [m][lane]; with the single
// layer alone the D_m slot holds the phase table e^{i l a}, l = 0..32, as [pair][33] double words,
// followed by rho^2 on the ring of every pair of the batch, [pair][Mt].
__host__ __device__ inline int64_t pair_scratch_per_warp(int L, bool withK, int Mt) {
  return withK ? (int64_t)2 * (L + 1) * 32 : (int64_t)(L + 1) * 32 + 2 * 33 * 32 + (int64_t)32 * Mt;
}

PairArgs make_pair_args(bie_surface s, double k, unsigned kernels);
bie_status launch_pairs(bie_surface s, PairArgs& a);

}  // namespace bie
