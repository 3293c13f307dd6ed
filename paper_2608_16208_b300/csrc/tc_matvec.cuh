// Tensor-core block matrix-vector product of the dense solve (tc_matvec.cu).
#pragma once
#include "bie_internal.cuh"

namespace bie {

// Split-BF16 image of an n x n complex matrix in the shared-memory layout of the MMA:
// [n_mt][n_kt][hi, lo][128 rows][128 bytes], plus a work image of the right-hand sides.
struct TcImage {
  int64_t n = 0;
  int n_mt = 0, n_kt = 0;   // row tiles of 128, k-tiles of 64 reals (32 complex columns)
  uint8_t* a_img = nullptr;
  uint8_t* b_img = nullptr; // [n_kt][hi, lo][32][128 bytes]
};

struct TcArgs {
  const uint8_t* a_img;
  const uint8_t* b_img;
  double2* y;
  int64_t ldy;
  int64_t n_rows;
  int nr;
  int n_mt, n_kt;
  int chunk;      // k-tiles accumulated in FP32 before the FP64 add
  int* status;    // status[1] set when a bounded wait expired
};

bie_status tc_image_create(bie_ctx ctx, int64_t n, const double* A, TcImage* out);
void tc_image_free(bie_ctx ctx, TcImage* im);
bie_status tc_matvec(bie_ctx ctx, TcImage& im, const double2* x, int64_t ldx, int nr, double2* y, int64_t ldy);

}  // namespace bie
