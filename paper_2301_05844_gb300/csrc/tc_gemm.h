// Task descriptor of the tcgen05 grouped GEMM (tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace bbp {

// C[m][n] = alpha * sum_k A[m][k] B[n][k]; A and B are read by TMA through the tensor maps
// (K innermost, rows outer, 128-byte swizzle, zero fill past the edges).  nseg = 3: split
// operands, each stored as two planes (hi, lo) with a map per plane; the GEMM runs three
// K-segments of K each, (A hi, B hi), (A lo, B hi), (A hi, B lo), accumulating
// A_hi B_hi + A_lo B_hi + A_hi B_lo.  Otherwise one segment through map_a, map_b.
// The result is written through the two-level map
//   C[(m/M2)*c_m1 + (m%M2)*c_m2 + (n/N2)*c_n1 + (n%N2)*c_n2]
// and, if C2 is set, also to C2 through (d_*).  out_kind: 0 FP32, 1 FP32 rounded to
// TF32, 2 BF16, 3 FP64.  x3 (bits 0-1 for C, 2-3 for C2): the destination is a split
// operand, hi in the first plane and lo kseg (kseg2) elements further.
struct TCTask {
    CUtensorMap map_a;
    CUtensorMap map_b;
    CUtensorMap map_a2;  // second (lo) planes of split operands
    CUtensorMap map_b2;
    int M, N, K, M2, N2, out_kind;
    long long c_m1, c_m2, c_n1, c_n2;
    long long d_m1, d_m2, d_n1, d_n2;
    void* C;
    void* C2;
    const int* active;
    float alpha;
    int x3;
    long long kseg, kseg2;
    int nseg;  // 3 for split operands, otherwise 1
};

cudaError_t tc_prepare();
// The operand ring holds stages of ksub k-blocks (1 or 2; 128 bytes of K each).  Deepest ring
// for tile width bn (0 for an unsupported ksub), and the planner's default depth (one k-block
// per stage) for a step of `kblocks` k-blocks.
int tc_max_stages(int bn, int ksub = 1);
int tc_default_stages(int bn, int kblocks);
// stages: depth of the shared-memory ring (1..tc_max_stages(bn, ksub)).  stall != 0 only in
// the self-test of the bounded waits: no operand is loaded, so a CTA's first wait runs out
// (or returns on the error another CTA raised), *err is raised and the launch ends.
cudaError_t launch_tc_gemm(const TCTask* d_tasks, int ntasks, int kind, int bn, int max_tiles, int stages, int* err,
                           cudaStream_t s, int ksub = 1, int stall = 0);
// kind: 0 FP32/TF32 elements, 1 BF16.  rows x K matrix with leading dimension ld_elems
// (ld * element size must be a multiple of 16 bytes, base 16-byte aligned).
cudaError_t tc_make_map(void* map_out, const void* base, int kind, long long rows, long long K, long long ld_elems,
                        int box_rows);

}  // namespace bbp
