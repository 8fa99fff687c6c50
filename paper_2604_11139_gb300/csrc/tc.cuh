// Tensor-core (tcgen05 / TMA) BF16-split GEMM interface (gemm_tc.cu).
#pragma once
#include <cuda_bf16.h>

#include "pw_internal.cuh"

namespace pw {
namespace tc {

enum TcEpiMode { TC_EPI_PARTIAL = 0, TC_EPI_ACCUM = 1, TC_EPI_CHEB = 2, TC_EPI_STORE = 3 };

// Output element (row r, column j) of the real view lives at base[j * ld + r].
struct TcEpi {
  int mode;
  // TC_EPI_PARTIAL: part[z * part_split_stride + j * part_ld + r] = acc (split z = blockIdx.z)
  float* part;
  int64_t part_ld, part_split_stride;
  // TC_EPI_ACCUM: out += alpha acc ; TC_EPI_STORE: out = alpha acc ;
  // TC_EPI_CHEB: out = alpha (out + acc - shift yk) - beta ykm1
  float* out;
  int64_t ldo;
  const float* yk;
  int64_t ldyk;
  const float* ykm1;
  int64_t ldykm1;
  float alpha, beta, shift;
  const double* dev_ce;  // optional device {c, e}: shift = c, alpha = (first ? 1 : 2) / e
  int first;
  // optional bf16 pieces of the CHEB output: split[p * split_piece_stride + j * split_ld + r]
  __nv_bfloat16* split;
  int64_t split_ld, split_piece_stride;
  int out_pieces;
};

// a K-major bf16 operand stored as pieces [pieces][rows][pitch] (pitch a multiple of 64)
struct Operand {
  const __nv_bfloat16* ptr;
  int64_t rows, pitch, piece_stride;
};

bool available();
// D (M x N) = sum over piece pairs of A (M x K) . B (N x K)^T, FP32 accumulation, then the epilogue.
// nsplit > 1 splits K (only meaningful with TC_EPI_PARTIAL).  *err (device) is set if a wait expired.
// test_no_copies: the producer issues no copies and every wait gives up after a few thousand
// polls, so the first wait expires and the failure path runs (failure-detection test).
cudaError_t gemm(const Operand& A, const Operand& B, int M, int N, int K, int pieces, int nsplit, const TcEpi& epi,
                 int* err, cudaStream_t st, int test_no_copies = 0);
int split_count(int K, int nsplit);
cudaError_t reduce_partials(const float* part, int nsplit, int64_t split_stride, int64_t part_ld, int M, int N,
                            float* out, int64_t ldo, cudaStream_t st);
cudaError_t split_f32(const float* x, int64_t ldx, int rows, int cols, int pieces, __nv_bfloat16* out, int64_t pitch,
                      int64_t piece_stride, cudaStream_t st);
cudaError_t build_a(const double2* P, int npw, int np, int pieces, __nv_bfloat16* A1, int64_t pitch1, int64_t ps1,
                    __nv_bfloat16* A2, int64_t pitch2, int64_t ps2, cudaStream_t st);

}  // namespace tc
}  // namespace pw
