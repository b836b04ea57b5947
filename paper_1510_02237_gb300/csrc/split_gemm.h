// split_gemm.h -- FP64-accurate tall-skinny products on the BF16 tensor cores
// (internal; not part of the public ABI).
//
// Every FP64 column x (of the basis Q, of a block V, of a coefficient block
// C) is written as x = 2^E * sum_{s=1..8} d_s 2^{-7 s} with a per-column
// exponent E (max |x| < 2^{E-1}) and integer digits |d_s| <= 64, which BF16
// holds exactly; the 8 digits leave x's remainder below 2^-55 max|x|.  A
// product sum_k x_k y_k then splits into the 43 digit products d_s e_t with
// s + t <= 10; products of equal s + t share one FP32 accumulator in TMEM.
// Each digit product is at most 2^12, so over a chunk of 256 contraction
// elements a group of at most 8 products sums to an integer below 2^23 --
// every partial sum is exact in FP32 whatever the summation order.  Chunk
// results are combined in FP64 (Horner in 2^-7), so the only errors are the
// digit remainders, the dropped digit products (s + t > 10, below
// 2^-58 max|x| max|y| per term) and the FP64 combination: the accuracy of an
// FP64 dot product, at the speed of the tensor cores and of HBM.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pr {

constexpr int SG_S = 8;         // digit slices per operand
constexpr int SG_N = 16;        // columns of the narrow operand per product
constexpr int SG_BM = 128;      // rows per tile (one TMEM lane each)
constexpr int SG_KC = 32;       // contraction elements per pipeline stage (64-byte rows)
constexpr int SG_L = 256;       // contraction elements per exact FP32 chunk

struct SplitGemm {
    long d = 0;                  // rows of Q (contraction length of Q^T V)
    int cap = 0, cap_pad = 0;    // basis capacity, padded to SG_KC
    int grid = 0;                // CTAs of the persistent product kernel (one per SM)
    // Digit slices in the tensor cores' operand layout: units of 8 rows x 32
    // contraction elements (512 bytes, 64-byte swizzle applied), ordered
    // [slice][contraction block][row group], so a 128-row operand tile of
    // one contraction block is 8 KB of consecutive memory.
    long nkb = 0;                  // contraction blocks of 32 over d
    int nlb = 0;                   // contraction blocks of 32 over cap_pad
    int ngl = 0;                   // row groups of 8 over cap_pad (basis columns)
    long ngd = 0;                  // row groups of 8 over d (state rows)
    __nv_bfloat16* Xc = nullptr;   // Q for Q^T V: rows = basis columns, contraction = state rows
    __nv_bfloat16* Xr = nullptr;   // Q for Q C: rows = state rows, contraction = basis columns
    __nv_bfloat16* Vs = nullptr;   // V (SG_N rows = its columns), contraction = state rows
    __nv_bfloat16* Cs = nullptr;   // 2^{E_l} C (SG_N rows), contraction = basis columns
    int* Eq = nullptr;             // [cap] column exponents of Q
    int* Fv = nullptr;             // [SG_N] column exponents of V
    int* Gc = nullptr;             // [SG_N] column exponents of 2^{E_l} C
    unsigned long long* Kq = nullptr;   // [cap_pad] column maxima keys (|x| bit patterns) of Q
    unsigned long long* Kv = nullptr;   // [SG_N] the same for V
    double* ws = nullptr;          // [grid][SG_N][cap_pad] partial sums of Q^T V
    double* C = nullptr;           // [SG_N][cap_pad] coefficients Q^T V (column-major, ld cap_pad)
    int* err = nullptr;            // sticky: a pipeline wait gave up
    // 4-D maps (element, row group, contraction block, digit slice): one load
    // brings all 8 slices of a stage's operand tile.  mapXc[i] / mapXr[i]
    // load 2 (i + 1) row groups (16 (i + 1) rows); mapVs / mapCs the 2 row
    // groups of the narrow operand.
    CUtensorMap mapXc[8], mapXr[8];
    CUtensorMap mapVs, mapCs;
    // With images (sg_init(..., true)): the basis images D = F(Q) - G(Q) in
    // the Xr layout, their column exponents, and the coefficient digits
    // folded with those exponents, so that z <- z - D C runs like v <- v - Q C.
    __nv_bfloat16* Dr = nullptr;
    __nv_bfloat16* CsD = nullptr;
    int* Ed = nullptr;             // [cap] column exponents of D
    int* GcD = nullptr;            // [SG_N] exponents of the folded coefficient columns
    unsigned long long* Kd = nullptr;   // [cap_pad] column maxima keys of D
    CUtensorMap mapDr[8], mapCsD;
};

// Bytes of device memory sg_init allocates for (d, cap, images).
size_t sg_bytes(long d, int cap, bool images = false);
// Allocate and set up (tensor maps included); d must be a multiple of 8;
// images: also hold the digits of the basis images D.
cudaError_t sg_init(SplitGemm* g, long d, int cap, bool images = false);
void sg_free(SplitGemm* g);
// Digits of columns [c0, c1) of Q in both layouts: a device range (c0_dev,
// c1_dev; at most maxcols <= SG_N columns) or host columns [c0_host,
// c0_host + maxcols).
cudaError_t sg_append(SplitGemm* g, const double* Q, long ldq, const int* c0_dev, const int* c1_dev, int c0_host,
                      int maxcols, cudaStream_t s);
// Digits of columns of D (the basis images), in the Xr layout, like sg_append.
cudaError_t sg_append_images(SplitGemm* g, const double* D, long ldd, const int* c0_dev, const int* c1_dev,
                             int c0_host, int maxcols, cudaStream_t s);
// z <- z - D C for the m <= SG_N image columns z (ld ldz), with the
// coefficients C of the last projection (g->C): the image update of a
// Gram-Schmidt pass.  Needs sg_init(..., true).
cudaError_t sg_update_images(SplitGemm* g, double* z, long ldz, int m, const int* r_dev, cudaStream_t s);
// One classical Gram-Schmidt pass of the m <= SG_N columns v (ld ldv) against
// Q[:, 0:*r_dev):  C = Q^T v (into g->C), then v <- v - Q C.
cudaError_t sg_cgs_pass(SplitGemm* g, double* v, long ldv, int m, const int* r_dev, cudaStream_t s);
// C = Q^T v only (g->C, ld cap_pad).
cudaError_t sg_project(SplitGemm* g, const double* v, long ldv, int m, const int* r_dev, cudaStream_t s);
// v <- v - Q C for a given coefficient block C (*r_dev x m, ld ldc).
cudaError_t sg_update(SplitGemm* g, double* v, long ldv, int m, const double* C, int ldc, const int* r_dev,
                      cudaStream_t s);

}  // namespace pr
