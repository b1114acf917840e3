// Tensor-core grouped GEMM for sm_103a (tcgen05 + TMEM + TMA).
//
//   C[m][n] = sum_k A[m][k] * B[n][k]      (A, B K-major; FP32 accumulation in TMEM)
//
// One CTA computes a 128 x BN tile of one task.  Warp 0 (one lane) streams A and B
// k-blocks with TMA into a ring of 2-8 stages of 128-byte-swizzled shared memory; warp 1
// (one lane) issues tcgen05.mma (kind::tf32 or kind::f16 with BF16 operands) into a
// TMEM accumulator; all four warps then read the accumulator with tcgen05.ld and
// scatter it through a two-level index map (the same map as the FP64 contraction),
// optionally to a second destination, rounding to TF32 or BF16 for the next GEMM.
//
// Every wait on an mbarrier is bounded: on timeout the CTA records an error in a
// device word, drains its own outstanding TMA copies (bounded), frees its TMEM and
// returns, so that a broken pipeline ends the launch with a status, not a hang.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "bbp_internal.h"
#include "tc_gemm.h"

namespace bbp {
namespace tc {

constexpr int BM = 128;
constexpr int STAGES = 8;  // deepest operand ring (mbarrier arrays); see tc_max_stages
constexpr int KBYTES = 128;  // bytes of K per k-block row (one 128-byte swizzle atom)
constexpr int KSUB_MAX = 2;  // k-blocks per ring stage: 1 or 2 (autotuned per step)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Programmatic dependent launch: wait for the previous kernel's completion (and its memory),
// and allow the next kernel to be scheduled.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Non-blocking test of a phase (a satisfied mbarrier.try_wait measured ~280 cycles on this
// GPU, a satisfied test_wait ~150; the waits below poll it in a bounded loop).
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok;
}
// Bounded wait for the phase with the given parity to complete.  Returns false (and
// raises *err) after ~2^22 polls, or immediately once another thread raised *err.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *(volatile int*)err) return false;
    }
    atomicExch(err, 1);
    return false;
}

// Bounded wait that ignores the error word: drains a CTA's own asynchronous work on the
// failure path (its copies and MMAs must finish before its shared memory and TMEM are
// released, whichever CTA raised the error).  Gives up after ~2^22 polls.
__device__ __forceinline__ bool mbar_wait_own(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void prefetch_map(const void* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int KIND>  // 0: tf32, 1: bf16 (kind::f16)
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;             // leading-dimension offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride-dimension offset: next 8-row group
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}
// Instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc(int kind, int bn) {
    return (1u << 4) | ((kind == 0 ? 2u : 1u) << 7) | ((kind == 0 ? 2u : 1u) << 10) | ((uint32_t)(bn >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void store_out(void* out, long long o, int kind, float x) {
    if (kind == 0) ((float*)out)[o] = x;
    else if (kind == 1) ((float*)out)[o] = round_tf32(x);
    else if (kind == 2) ((__nv_bfloat16*)out)[o] = __float2bfloat16_rn(x);
    else ((double*)out)[o] = (double)x;
}

// Epilogue.  The accumulator is staged in shared memory 64 columns at a time as FP32
// [BM][EC+1] (odd row pitch: row-wise and column-wise accesses are both free of bank
// conflicts), and each chunk is written to each destination through the two-level index
// map, with the row and column offsets (m1*sm1 + m2*sm2, n1*sn1 + n2*sn2) computed once
// per chunk.  A destination that is
// contiguous along n2 is written row by row, one 16-byte vector per thread (a warp covers
// up to 32 vectors of one row); one contiguous along m2 is written column by column in
// 16-byte vectors down the rows; any other map falls back to element stores.  A vector is
// used only where its elements are contiguous and 16-byte aligned in the destination.
__device__ __forceinline__ int out_esz(int kind) { return kind == 3 ? 8 : kind == 2 ? 2 : 4; }

__device__ __forceinline__ void store_vec(void* out, long long o, int kind, const float* x) {
    // element o of out starts a 16-byte-aligned run of 16 / element-size elements
    if (kind == 2) {
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
        *(uint4*)((__nv_bfloat16*)out + o) = *(const uint4*)h;
    } else if (kind == 3) {
        *(double2*)((double*)out + o) = make_double2((double)x[0], (double)x[1]);
    } else if (kind == 1) {
        *(float4*)((float*)out + o) = make_float4(round_tf32(x[0]), round_tf32(x[1]), round_tf32(x[2]), round_tf32(x[3]));
    } else {
        *(float4*)((float*)out + o) = make_float4(x[0], x[1], x[2], x[3]);
    }
}

constexpr int EC = 64;  // epilogue chunk (columns)
// Staged rows are skewed by one slot per 32 rows: row r lives at slot r + r / 32 (pitch EC + 1),
// so that the 16 lanes reading rows 8l + j of one column (a vector down a column) hit 16
// different banks, while row-wise and lane-per-row accesses stay conflict-free.
constexpr int TROWS = BM + BM / 32;
__device__ __forceinline__ int trow(int r) { return r + (r >> 5); }

// Split destination (x3 != 0): two planes kseg elements apart, hi = r(x) in the first and
// lo = r(x - hi) in the second, r the rounding of the element kind (TF32 for kind 1, BF16 for
// kind 2); x - hi is exact in FP32 for both.  A consumer GEMM reads the planes of an A operand
// in the K-segment order (hi, lo, hi) and those of a B operand as (hi, hi, lo).
__device__ __forceinline__ void store_split1(void* out, long long o, int kind, float x, long long kseg) {
    if (kind == 2) {
        const __nv_bfloat16 hb = __float2bfloat16_rn(x);
        const __nv_bfloat16 lb = __float2bfloat16_rn(x - __bfloat162float(hb));
        __nv_bfloat16* b = (__nv_bfloat16*)out;
        b[o] = hb;
        b[o + kseg] = lb;
        return;
    }
    float* f = (float*)out;
    const float hi = round_tf32(x), lo = round_tf32(x - hi);
    f[o] = hi;
    f[o + kseg] = lo;
}
// 16 bytes per plane: 4 TF32 elements (kind 1) or 8 BF16 elements (kind 2)
__device__ __forceinline__ void store_split_vec(void* out, long long o, int kind, const float* x, long long kseg) {
    if (kind == 2) {
        __nv_bfloat162 h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
            const float2 hf = __bfloat1622float2(h[j]);
            l[j] = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
        }
        __nv_bfloat16* b = (__nv_bfloat16*)out;
        *(uint4*)(b + o) = *(const uint4*)h;
        *(uint4*)(b + o + kseg) = *(const uint4*)l;
        return;
    }
    float hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        hi[j] = round_tf32(x[j]);
        lo[j] = round_tf32(x[j] - hi[j]);
    }
    float* f = (float*)out;
    *(float4*)(f + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    *(float4*)(f + o + kseg) = make_float4(lo[0], lo[1], lo[2], lo[3]);
}

// The epilogue runs on the EPI_THREADS threads of EPI_THREADS / 32 epilogue warps: eight of
// them drain the TMEM accumulator into the staged tile (two per quarter of the TMEM lanes), all
// of them write the staged tile out (the stores are latency-bound, so more warps hide more of
// it).  They synchronise among themselves on named barrier 1.
constexpr int EPI_THREADS = 512;
constexpr int DRAIN_WARPS = 8;
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory"); }
// the same barrier, returning whether every epilogue thread passed true
__device__ __forceinline__ bool epi_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(EPI_THREADS)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void epilogue_dest(const float* tile, long long* roff, long long* coff, int rows, int ncols,
                                              int m0, int n0, int M2, int N2, long long sm1, long long sm2,
                                              long long sn1, long long sn2, int kind, float alpha, void* out, int x3,
                                              long long kseg, int tid) {
    constexpr int P = EC + 1;
    epi_sync();  // the previous destination has finished with the offsets
    for (int r = tid; r < rows; r += EPI_THREADS) {
        const int m = m0 + r, m1 = m / M2;
        roff[r] = (long long)m1 * sm1 + (long long)(m - m1 * M2) * sm2;
    }
    for (int c = tid; c < ncols; c += EPI_THREADS) {
        const int n = n0 + c, n1 = n / N2;
        coff[c] = (long long)n1 * sn1 + (long long)(n - n1 * N2) * sn2;
    }
    epi_sync();
    const int esz = out_esz(kind), VW = 16 / esz;
    const uintptr_t base = (uintptr_t)out;
    // a split destination vectorises only if its second plane starts 16-byte aligned as well
    const bool segs_aligned = !x3 || ((kseg * esz) & 15) == 0;
    float x[8];
    // fully regular destinations (below): every group of VW rows (columns) is one vector
    const bool al = (base & 15) == 0 && segs_aligned;
    const bool vec_m = al && sm2 == 1 && M2 % VW == 0 && m0 % VW == 0 && sm1 % VW == 0 && sn1 % VW == 0 && sn2 % VW == 0;
    const bool vec_n = !vec_m && al && sn2 == 1 && N2 % VW == 0 && n0 % VW == 0 && sn1 % VW == 0 && sm1 % VW == 0 &&
                       sm2 % VW == 0;
    // A destination whose contiguous runs cannot line up with vectors (split segments not
    // 16-byte aligned: the site-update operands of D=5, whose segments are K = 625 apart; or a
    // run length that is no multiple of the vector width, such as q = 25) takes no vector at
    // all: one pass of scalar stores, each warp on one row (one column) at a time with its
    // lanes on consecutive destination addresses, no per-element test or index division.
    if (!vec_m && !vec_n && (!segs_aligned || (sn2 == 1 && N2 % VW) || (sm2 == 1 && M2 % VW)) &&
        (sn2 == 1 || sm2 == 1)) {
        const int wq = tid >> 5, ln = tid & 31;
        constexpr int NW = EPI_THREADS / 32;
        if (sn2 == 1) {
            for (int r = wq; r < rows; r += NW) {
                const long long ro = roff[r];
                for (int c = ln; c < ncols; c += 32) {
                    const float xv = tile[trow(r) * P + c] * alpha;
                    if (x3) store_split1(out, ro + coff[c], kind, xv, kseg);
                    else store_out(out, ro + coff[c], kind, xv);
                }
            }
        } else {
            for (int c = wq; c < ncols; c += NW) {
                const long long co = coff[c];
                for (int r = ln; r < rows; r += 32) {
                    const float xv = tile[trow(r) * P + c] * alpha;
                    if (x3) store_split1(out, roff[r] + co, kind, xv, kseg);
                    else store_out(out, roff[r] + co, kind, xv);
                }
            }
        }
        return;
    }
    // Fully regular destinations: contiguous along m2 (or n2) in runs that are whole multiples
    // of the vector width, every run start and segment 16-byte aligned.  Then every group of VW
    // rows (columns) of the chunk is one vector: a single pass, no per-group test; lanes run
    // along the contiguous direction (consecutive 16-byte stores), a ragged tail in scalars.
    if (vec_m) {
        const int G = rows / VW;
        for (int it = tid; it < ncols * G; it += EPI_THREADS) {
            const int c = it / G, r0 = (it - c * G) * VW;
            const long long o = roff[r0] + coff[c];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < VW) x[j] = tile[trow(r0 + j) * P + c] * alpha;
            if (x3) store_split_vec(out, o, kind, x, kseg);
            else store_vec(out, o, kind, x);
        }
        for (int it = tid; it < ncols * (rows - G * VW); it += EPI_THREADS) {
            const int c = it / (rows - G * VW), r = G * VW + it % (rows - G * VW);
            const float xv = tile[trow(r) * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
        return;
    }
    if (vec_n) {
        const int G = ncols / VW;
        for (int it = tid; it < rows * G; it += EPI_THREADS) {
            const int r = it / G, c0 = (it - r * G) * VW;
            const long long o = roff[r] + coff[c0];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < VW) x[j] = tile[trow(r) * P + c0 + j] * alpha;
            if (x3) store_split_vec(out, o, kind, x, kseg);
            else store_vec(out, o, kind, x);
        }
        for (int it = tid; it < rows * (ncols - G * VW); it += EPI_THREADS) {
            const int r = it / (ncols - G * VW), c = G * VW + it % (ncols - G * VW);
            const float xv = tile[trow(r) * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
        return;
    }
    // Otherwise two passes: 16-byte vectors where a group of VW elements is contiguous and
    // aligned in the destination, then every other element with consecutive lanes on
    // consecutive destination addresses (so that a warp's scalar stores share a few sectors).
    if (sn2 == 1) {
        const int G = (ncols + VW - 1) / VW;
        auto is_vec = [&](int r, int c0) {
            const long long o = roff[r] + coff[c0];
            return segs_aligned && c0 + VW <= ncols && ((base + (uintptr_t)(o * esz)) & 15) == 0 &&
                   coff[c0 + VW - 1] == coff[c0] + VW - 1;
        };
        for (int it = tid; it < rows * G; it += EPI_THREADS) {
            const int r = it / G, c0 = (it - r * G) * VW;
            if (!is_vec(r, c0)) continue;
            const long long o = roff[r] + coff[c0];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < VW) x[j] = tile[trow(r) * P + c0 + j] * alpha;
            if (x3) store_split_vec(out, o, kind, x, kseg);
            else store_vec(out, o, kind, x);
        }
        for (int it = tid; it < rows * ncols; it += EPI_THREADS) {  // lanes along a row
            const int r = it / ncols, c = it - r * ncols;
            if (is_vec(r, c - c % VW)) continue;
            const float xv = tile[trow(r) * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
    } else if (sm2 == 1) {
        const int G = (rows + VW - 1) / VW;
        auto is_vec = [&](int r0, int c) {
            const long long o = roff[r0] + coff[c];
            return segs_aligned && r0 + VW <= rows && ((base + (uintptr_t)(o * esz)) & 15) == 0 &&
                   roff[r0 + VW - 1] == roff[r0] + VW - 1;
        };
        for (int it = tid; it < ncols * G; it += EPI_THREADS) {
            const int c = it / G, r0 = (it - c * G) * VW;
            if (!is_vec(r0, c)) continue;
            const long long o = roff[r0] + coff[c];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < VW) x[j] = tile[trow(r0 + j) * P + c] * alpha;
            if (x3) store_split_vec(out, o, kind, x, kseg);
            else store_vec(out, o, kind, x);
        }
        for (int it = tid; it < rows * ncols; it += EPI_THREADS) {  // lanes down a column
            const int c = it / rows, r = it - c * rows;
            if (is_vec(r - r % VW, c)) continue;
            const float xv = tile[trow(r) * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
    } else {
        for (int it = tid; it < rows * ncols; it += EPI_THREADS) {
            const int c = it / rows, r = it - c * rows;
            const float xv = tile[trow(r) * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
    }
}

constexpr int EPI_WARPS = EPI_THREADS / 32;      // warps 2..; 2..9 drain TMEM, two per lane quarter
constexpr int NTHREADS = 32 * (2 + EPI_WARPS);   // producer, MMA issuer, epilogue
constexpr size_t EPI_BYTES = (size_t)TROWS * (EC + 1) * sizeof(float) + (size_t)(BM + EC) * sizeof(long long);

// Persistent, warp-specialised grouped GEMM.  The work items of a launch are the tiles of all
// its tasks (task = item / max_tiles, tile = item % max_tiles; tiles a task does not have are
// skipped, and so are the tasks whose active flag is 0); CTA b takes items b, b + G, b + 2G, ...
// Warp 0 (one lane) streams the k-blocks of its items through a ring of stages with TMA, warp 1
// (one lane) issues the MMAs of item j into TMEM accumulator j & 1, and warps 2-9 drain the
// other accumulator meanwhile (two warps per quarter of the TMEM lanes, alternate 16-column
// groups): the epilogue of one tile runs under the loads and MMAs of the next.  The tiles of one row block are consecutive items (their A rows reach L2 once).
// stall != 0 (self-test of the bounded waits only): the producer issues no copy, so the
// first wait on a full stage never succeeds and must end by its bound.
template <int KIND, int BN>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc_gemm(const TCTask* __restrict__ tasks, int ntasks, int max_tiles,
                                                         int* err, int stages, int ksub, int stall) {
    constexpr int EK = KBYTES / (KIND == 0 ? 4 : 2);  // elements of K per k-block
    constexpr uint32_t A_BYTES = BM * KBYTES, B_BYTES = BN * KBYTES;  // one k-block
    constexpr uint32_t TCOLS = 2 * (BN < 32 ? 32 : BN);               // two accumulators
    const uint32_t A_STAGE = A_BYTES * ksub, B_STAGE = B_BYTES * ksub;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // aligned to 1024 bytes by pointer arithmetic on the shared array (an integer round trip
    // would turn every access through these pointers into a generic one)
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA = smem;
    unsigned char* sB = smem + stages * A_STAGE;
    float* tile = (float*)(sB + stages * B_STAGE);  // epilogue staging, its own region
    long long* roff = (long long*)(tile + TROWS * (EC + 1));
    long long* coff = roff + BM;
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ int issued;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], DRAIN_WARPS);
        }
        mbar_init(&mma_done, 1);
        issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, TCOLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    // Everything above reads no earlier kernel's output, so it may overlap the previous kernel
    // (programmatic dependent launch); the active flags and the operands are its output.
    grid_dependency_wait();
    const int nitems = ntasks * max_tiles;
    // item -> (task, m0, n0), or false if the item is empty (same answer in every role)
    auto item = [&](int w, const TCTask*& t, int& m0, int& n0) {
        t = tasks + w / max_tiles;
        const int tl = w % max_tiles;
        const int tilesM = (t->M + BM - 1) / BM, tilesN = (t->N + BN - 1) / BN;
        if (tl >= tilesM * tilesN) return false;
        if (t->active && *t->active == 0) return false;
        n0 = (tl % tilesN) * BN;
        m0 = (tl / tilesN) * BM;
        return true;
    };

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: stage gks holds k-blocks of one item (the last stage may hold fewer)
            int gks = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok && !stall; w += gridDim.x) {
                const TCTask* t;
                int m0, n0;
                if (!item(w, t, m0, n0)) continue;
                prefetch_map(&t->map_a);
                prefetch_map(&t->map_b);
                const int nk1 = (t->K + EK - 1) / EK;  // k-blocks of one K-segment
                const int nseg = t->nseg == 3 ? 3 : 1;
                if (nseg == 3) {
                    prefetch_map(&t->map_a2);
                    prefetch_map(&t->map_b2);
                }
                const int nk = nk1 * nseg, nst = (nk + ksub - 1) / ksub;
                for (int ks = 0; ks < nst; ++ks, ++gks) {
                    const int s = gks % stages, r = gks / stages;
                    if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1, err)) {
                        ok = false;
                        break;
                    }
                    const int na = min(ksub, nk - ks * ksub);
                    mbar_expect_tx(&full[s], (uint32_t)na * (A_BYTES + B_BYTES));
                    for (int a = 0; a < na; ++a) {
                        // split operands: segment 0 = (A hi, B hi), 1 = (A lo, B hi), 2 = (A hi, B lo);
                        // a segment's last k-block reads past K, which the maps fill with zeros
                        const int kb = ks * ksub + a, seg = kb / nk1, kk = kb - seg * nk1;
                        tma_load_2d(sA + s * A_STAGE + a * A_BYTES, seg == 1 ? &t->map_a2 : &t->map_a, &full[s], kk * EK, m0);
                        tma_load_2d(sB + s * B_STAGE + a * B_BYTES, seg == 2 ? &t->map_b2 : &t->map_b, &full[s], kk * EK, n0);
                    }
                    issued = gks + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: item j into accumulator j & 1, once the epilogue has emptied it
            constexpr uint32_t ID = idesc(KIND, BN);
            int gks = 0, j = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
                const TCTask* t;
                int m0, n0;
                if (!item(w, t, m0, n0)) continue;
                const int b = j & 1, u = j >> 1;
                if (u > 0 && !mbar_wait(&tempty[b], (u - 1) & 1, err)) break;
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * (TCOLS / 2));
                const int nk = ((t->K + EK - 1) / EK) * (t->nseg == 3 ? 3 : 1), nst = (nk + ksub - 1) / ksub;
                for (int ks = 0; ks < nst; ++ks, ++gks) {
                    const int s = gks % stages, r = gks / stages;
                    if (!mbar_wait(&full[s], r & 1, err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const int na = min(ksub, nk - ks * ksub);
                    for (int a = 0; a < na; ++a) {
                        const int kb = ks * ksub + a;
                        const uint32_t a0 = smem_u32(sA + s * A_STAGE + a * A_BYTES);
                        const uint32_t b0 = smem_u32(sB + s * B_STAGE + a * B_BYTES);
#pragma unroll
                        for (int k = 0; k < KBYTES / 32; ++k)  // 32 bytes of K per instruction
                            umma<KIND>(acc, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), ID, (kb | k) ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&tfull[b]);
                ++j;
            }
            umma_commit(&mma_done);  // completes once every MMA issued above has
        }
    } else {
        // epilogue: item j from accumulator j & 1, 64 columns at a time through shared memory
        const int etid = threadIdx.x - 64;            // 0..EPI_THREADS-1
        const bool drains = warp < 2 + DRAIN_WARPS;   // warps 2..9 read the accumulator
        const int quad = warp & 3;                    // TMEM lanes 32 quad .. 32 quad + 31
        const int half = (warp - 2) >> 2;             // this warp's 16-column groups: c / 16 = half mod 2
        const int row = quad * 32 + lane;
        int j = 0;
        for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
            const TCTask* t;
            int m0, n0;
            if (!item(w, t, m0, n0)) continue;
            const int b = j & 1, u = j >> 1;
            if (w + (int)gridDim.x >= nitems) launch_dependents();  // the last item of this CTA
            // one decision for all epilogue warps, so that none is left at a barrier
            if (!epi_all(mbar_wait(&tfull[b], u & 1, err))) break;
            fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * (TCOLS / 2)) + ((uint32_t)(quad * 32) << 16);
            const int ncols = min(BN, t->N - n0), rows = min(BM, t->M - m0);
#pragma unroll 1
            for (int c0 = 0; c0 < ncols; c0 += EC) {
                const int cn = min(EC, ncols - c0);
                const int nchunk = (cn + 15) & ~15;  // tcgen05.ld is warp-collective: uniform bound
                epi_sync();                          // the previous chunk has been written out
                if (drains) {
                    // this warp's two 16-column groups of the chunk: both loads issued, one wait
                    const int c = 16 * half;
                    uint32_t v[16], w[16];
                    const bool two = c + 32 < nchunk;  // uniform: nchunk is
                    if (c < nchunk) tmem_ld16_issue(acc + (uint32_t)(c0 + c), v);
                    if (two) tmem_ld16_issue(acc + (uint32_t)(c0 + c + 32), w);
                    tmem_wait_ld();
                    float* trw = tile + trow(row) * (EC + 1);
                    if (c < nchunk) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) trw[c + q] = __uint_as_float(v[q]);
                    }
                    if (two) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) trw[c + 32 + q] = __uint_as_float(w[q]);
                    }
                }
                if (drains && c0 + EC >= ncols) {  // every column of this accumulator has been read
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
                for (int dst = 0; dst < (t->C2 ? 2 : 1); ++dst) {
                    void* out = dst ? t->C2 : t->C;
                    const long long sm1 = dst ? t->d_m1 : t->c_m1, sm2 = dst ? t->d_m2 : t->c_m2;
                    const long long sn1 = dst ? t->d_n1 : t->c_n1, sn2 = dst ? t->d_n2 : t->c_n2;
                    const int x3 = (t->x3 >> (2 * dst)) & 3;
                    epilogue_dest(tile, roff, coff, rows, cn, m0, n0 + c0, t->M2, t->N2, sm1, sm2, sn1, sn2,
                                  t->out_kind, t->alpha, out, x3, dst ? t->kseg2 : t->kseg, etid);
                }
            }
            ++j;
        }
    }
    __syncthreads();
    // drain after a failed wait (here or in another CTA): the MMAs issued must have finished
    // before TMEM is released, and the producer's copies must have landed before the CTA exits
    // (its shared memory may be given to the next CTA).  mma_done is committed after the MMA
    // loop in every case; these waits ignore the error word and have their own bound.
    if (threadIdx.x == 0 && *(volatile int*)err) {
        mbar_wait_own(&mma_done, 0);
        const int n_issued = issued;
        for (int g = (n_issued > stages ? n_issued - stages : 0); g < n_issued; ++g)
            mbar_wait_own(&full[g % stages], (g / stages) & 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

}  // namespace tc

// Dynamic shared memory: the operand ring, or the staged epilogue tile and its offsets
// if that is larger, plus 1 KB for the 1024-byte alignment of the swizzled ring.
// Dynamic shared memory: the operand ring and the epilogue's staging tile with its offsets,
// plus 1 KB for the 1024-byte alignment of the swizzled ring.
static size_t tc_smem(int stages, int bn, int ksub) {
    const size_t ring = (size_t)stages * (tc::BM + bn) * tc::KBYTES * ksub;
    return ring + tc::EPI_BYTES + 1024;
}

// Deepest ring (stages of ksub k-blocks) that fits, next to the epilogue's staging tile, the
// 227 KB of shared memory a CTA may hold (2 KB kept for the static barriers).
int tc_max_stages(int bn, int ksub) {
    if (ksub < 1 || ksub > tc::KSUB_MAX) return 0;
    const size_t per = (size_t)(tc::BM + bn) * tc::KBYTES * ksub;
    const size_t cap = 232448 - 2048 - 1024 - tc::EPI_BYTES;
    return std::max(1, std::min(tc::STAGES, (int)(cap / per)));
}

// Default ring depth (one k-block per stage): up to 4 stages, at least 2, at most the stages
// the K extent needs and the shared memory holds.
int tc_default_stages(int bn, int kblocks) {
    return std::max(1, std::min(std::min(kblocks, 4), tc_max_stages(bn, 1)));
}

static int tc_sm_count() {
    static std::atomic<int> cached{0};  // read by the server's worker and read-out threads
    int n = cached.load(std::memory_order_relaxed);
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cached.store(n, std::memory_order_relaxed);
    }
    return n;
}

cudaError_t tc_prepare() {
    // sets the shared-memory limits outside any stream capture
    cudaError_t e;
    const int bns[4] = {32, 64, 128, 256};
    for (int i = 0; i < 4; ++i) {
        const size_t smem = std::max(tc_smem(tc_max_stages(bns[i], 1), bns[i], 1), tc_smem(tc_max_stages(bns[i], 2), bns[i], 2));
        switch (bns[i]) {
            case 32:
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<0, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                break;
            case 64:
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<0, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<1, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                break;
            case 128:
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                break;
            default:
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<0, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
                if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_tc_gemm(const TCTask* d_tasks, int ntasks, int kind, int bn, int max_tiles, int stages, int* err,
                           cudaStream_t s, int ksub, int stall) {
    if (ntasks <= 0) return cudaSuccess;
    if (ksub < 1) ksub = 1;
    if (stages < 1 || stages > tc_max_stages(bn, ksub)) return cudaErrorInvalidValue;
    const size_t smem = tc_smem(stages, bn, ksub);
    // persistent CTAs: as many as fit on the GPU at once, never more than the work items
    const long long items = (long long)ntasks * max_tiles;
    const int per_sm = std::max(1, std::min(4, (int)((233472 - 2048) / (smem + 2048))));
    const int grid = (int)std::max(1LL, std::min(items, (long long)tc_sm_count() * per_sm));
    // programmatic dependent launch: the kernel waits (griddepcontrol.wait) before it reads
    // anything an earlier kernel wrote
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tc::NTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define TC_CASE(K_, N_)                                                                                        \
    if (kind == K_ && bn == N_)                                                                                \
        return cudaLaunchKernelEx(&cfg, tc::k_tc_gemm<K_, N_>, d_tasks, ntasks, max_tiles, err, stages, ksub, stall);
    TC_CASE(0, 32) TC_CASE(0, 64) TC_CASE(0, 128) TC_CASE(0, 256)
    TC_CASE(1, 32) TC_CASE(1, 64) TC_CASE(1, 128) TC_CASE(1, 256)
#undef TC_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- host: tensor maps
// The CUDA driver's tensor-map encoder (cuTensorMapEncodeTiled), looked up once (the request server encodes maps from its
// worker and read-out threads).
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? (PFN_cuTensorMapEncodeTiled_v12000)p : nullptr;
    }();
    return fn;
}

cudaError_t tc_make_map(void* map_out, const void* base, int kind, long long rows, long long K, long long ld_elems,
                        int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 g_encode = encoder();
    if (!g_encode) return cudaErrorNotSupported;
    const int esz = kind == 0 ? 4 : 2;
    cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)(ld_elems * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(tc::KBYTES / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode((CUtensorMap*)map_out, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          2, const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace bbp
