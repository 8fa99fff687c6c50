// FP64-accurate complex GEMM on the bf16 tensor cores (zgemm_tc.cu).
#pragma once
#include <cuda_bf16.h>

#include "pw_internal.cuh"

namespace pw {
namespace oz {

constexpr int kDigits = 7;  // 7-bit digits per operand entry (49 bits of each row-scaled entry)

// Digit planes of a K-major realified operand: dig[s * plane + row * pitch + k], s < kDigits,
// rows x k2 bf16 values (k2 = 2 x complex K), and one power-of-two exponent per complex row
// (A form) or per column (B form): entry = 2^exp * sum_s digit_s 2^(-7 (s + 1)).
struct Digits {
  const __nv_bfloat16* dig;
  int rows;       // realified rows: 2 x complex rows (A form) or columns of op(B) (B form)
  int k2;         // realified K
  int64_t pitch;  // elements per row (multiple of 8)
  int64_t plane;  // elements per digit plane
  const int* exp;
};

// Bytes of digit planes for `rows` realified rows of realified length k2.
size_t digit_bytes(int rows, int k2);
int64_t digit_pitch(int k2);

// Slices op(X) (R x K complex; element (r, l) = X[r * sr + l * sl], conjugated if cj) into digit
// planes: A form (aform != 0) gives the real matrix of 2R rows [Re -Im; Im Re] per complex
// entry, B form gives R rows of interleaved (Re, Im) along K.  amax: R scratch words.
cudaError_t slice(const double2* X, int64_t sr, int64_t sl, int cj, int R, int K, int aform, __nv_bfloat16* dig,
                  int64_t pitch, int64_t plane, unsigned long long* amax, int* exp, cudaStream_t st);

// Split count of a GEMM with realified M2 x N output over realified K k2 (whole K chunks).
int split_count(int M2, int N, int k2, int lower);

// C (M x N complex) = op(A) op(B) with the epilogue `epi`: A in A form (rows 2M), B in B form
// (rows N), both of realified length 2K.  lower != 0: only the 64 x 64 complex tiles on or
// below the diagonal (M == N).  nsplit > 1 reduces through `part` (nsplit * N * 2M doubles).
// *err (device) is set if a bounded wait expired; test_no_copies makes the producer issue no
// copies with a short wait limit, so that the first wait expires (failure-path test).
cudaError_t gemm(const Digits& A, const Digits& B, int M, int N, int K, const Epi<double>& epi, int lower,
                 int nsplit, double* part, int* err, int test_no_copies, cudaStream_t st);

bool available();

}  // namespace oz
}  // namespace pw
