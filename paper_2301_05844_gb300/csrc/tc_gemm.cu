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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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

// Split destination (x3 = 1: A rows [hi|lo|hi], 2: B rows [hi|hi|lo], segments kseg
// elements apart): hi = r(x), lo = r(x - hi), r the rounding of the element kind (TF32 for
// kind 1, BF16 for kind 2); x - hi is exact in FP32 for both.
__device__ __forceinline__ void store_split1(void* out, long long o, int kind, float x, int x3, long long kseg) {
    if (kind == 2) {
        const __nv_bfloat16 hb = __float2bfloat16_rn(x);
        const __nv_bfloat16 lb = __float2bfloat16_rn(x - __bfloat162float(hb));
        __nv_bfloat16* b = (__nv_bfloat16*)out;
        b[o] = hb;
        b[o + kseg] = x3 == 1 ? lb : hb;
        b[o + 2 * kseg] = x3 == 1 ? hb : lb;
        return;
    }
    float* f = (float*)out;
    const float hi = round_tf32(x), lo = round_tf32(x - hi);
    f[o] = hi;
    f[o + kseg] = x3 == 1 ? lo : hi;
    f[o + 2 * kseg] = x3 == 1 ? hi : lo;
}
// 16 bytes per segment: 4 TF32 elements (kind 1) or 8 BF16 elements (kind 2)
__device__ __forceinline__ void store_split_vec(void* out, long long o, int kind, const float* x, int x3,
                                                long long kseg) {
    uint4 H, Lo;
    if (kind == 2) {
        __nv_bfloat162 h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
            const float2 hf = __bfloat1622float2(h[j]);
            l[j] = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
        }
        H = *(const uint4*)h;
        Lo = *(const uint4*)l;
        __nv_bfloat16* b = (__nv_bfloat16*)out;
        *(uint4*)(b + o) = H;
        *(uint4*)(b + o + kseg) = x3 == 1 ? Lo : H;
        *(uint4*)(b + o + 2 * kseg) = x3 == 1 ? H : Lo;
        return;
    }
    float hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        hi[j] = round_tf32(x[j]);
        lo[j] = round_tf32(x[j] - hi[j]);
    }
    float* f = (float*)out;
    const float4 Hf = make_float4(hi[0], hi[1], hi[2], hi[3]), Lf = make_float4(lo[0], lo[1], lo[2], lo[3]);
    *(float4*)(f + o) = Hf;
    *(float4*)(f + o + kseg) = x3 == 1 ? Lf : Hf;
    *(float4*)(f + o + 2 * kseg) = x3 == 1 ? Hf : Lf;
}

__device__ __forceinline__ void epilogue_dest(const float* tile, long long* roff, long long* coff, int rows, int ncols,
                                              int m0, int n0, int M2, int N2, long long sm1, long long sm2,
                                              long long sn1, long long sn2, int kind, float alpha, void* out, int x3,
                                              long long kseg) {
    constexpr int P = EC + 1;
    const int tid = threadIdx.x;
    __syncthreads();  // the previous destination has finished with the offsets
    for (int r = tid; r < rows; r += 128) {
        const int m = m0 + r, m1 = m / M2;
        roff[r] = (long long)m1 * sm1 + (long long)(m - m1 * M2) * sm2;
    }
    for (int c = tid; c < ncols; c += 128) {
        const int n = n0 + c, n1 = n / N2;
        coff[c] = (long long)n1 * sn1 + (long long)(n - n1 * N2) * sn2;
    }
    __syncthreads();
    const int esz = out_esz(kind), VW = 16 / esz;
    const uintptr_t base = (uintptr_t)out;
    // a split destination vectorises only if every segment start stays 16-byte aligned
    const bool segs_aligned = !x3 || ((kseg * esz) & 15) == 0;
    float x[8];
    // Two passes per destination: 16-byte vectors where a group of VW elements is contiguous
    // and aligned in the destination, then every other element with consecutive lanes on
    // consecutive destination addresses (so that a warp's scalar stores share a few sectors:
    // the site-update operands of D=5 have contiguous runs of K = 25 elements, and split rows
    // whose segments are K apart, neither of which is 16-byte aligned).
    if (sn2 == 1) {
        const int G = (ncols + VW - 1) / VW;
        auto is_vec = [&](int r, int c0) {
            const long long o = roff[r] + coff[c0];
            return segs_aligned && c0 + VW <= ncols && ((base + (uintptr_t)(o * esz)) & 15) == 0 &&
                   coff[c0 + VW - 1] == coff[c0] + VW - 1;
        };
        for (int it = tid; it < rows * G; it += 128) {
            const int r = it / G, c0 = (it - r * G) * VW;
            if (!is_vec(r, c0)) continue;
            const long long o = roff[r] + coff[c0];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < VW) x[j] = tile[r * P + c0 + j] * alpha;
            if (x3) store_split_vec(out, o, kind, x, x3, kseg);
            else store_vec(out, o, kind, x);
        }
        for (int it = tid; it < rows * ncols; it += 128) {  // lanes along a row
            const int r = it / ncols, c = it - r * ncols;
            if (is_vec(r, c - c % VW)) continue;
            const float xv = tile[r * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, x3, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
    } else if (sm2 == 1) {
        const int G = (rows + VW - 1) / VW;
        auto is_vec = [&](int r0, int c) {
            const long long o = roff[r0] + coff[c];
            return segs_aligned && r0 + VW <= rows && ((base + (uintptr_t)(o * esz)) & 15) == 0 &&
                   roff[r0 + VW - 1] == roff[r0] + VW - 1;
        };
        for (int it = tid; it < ncols * G; it += 128) {
            const int c = it / G, r0 = (it - c * G) * VW;
            if (!is_vec(r0, c)) continue;
            const long long o = roff[r0] + coff[c];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < VW) x[j] = tile[(r0 + j) * P + c] * alpha;
            if (x3) store_split_vec(out, o, kind, x, x3, kseg);
            else store_vec(out, o, kind, x);
        }
        for (int it = tid; it < rows * ncols; it += 128) {  // lanes down a column
            const int c = it / rows, r = it - c * rows;
            if (is_vec(r - r % VW, c)) continue;
            const float xv = tile[r * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, x3, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
    } else {
        for (int it = tid; it < rows * ncols; it += 128) {
            const int c = it / rows, r = it - c * rows;
            const float xv = tile[r * P + c] * alpha;
            if (x3) store_split1(out, roff[r] + coff[c], kind, xv, x3, kseg);
            else store_out(out, roff[r] + coff[c], kind, xv);
        }
    }
}

template <int KIND, int BN>
// stall != 0 (self-test of the bounded waits only): the producer issues no copy, so the
// first wait on a full stage never succeeds and must end by its bound.
__global__ void __launch_bounds__(128, 1) k_tc_gemm(const TCTask* __restrict__ tasks, int* err, int stages, int ksub,
                                                    int stall) {
    // The task descriptor is copied to shared memory in one coalesced read (its fields are
    // otherwise fetched from global memory one dependent load at a time); the TMA copies use
    // the tensor maps at their global address.
    __shared__ TCTask t;
    const TCTask* gt = tasks + blockIdx.y;
    for (int w = threadIdx.x; w < (int)(sizeof(TCTask) / 4); w += 128)
        ((uint32_t*)&t)[w] = ((const uint32_t*)gt)[w];
    __syncthreads();
    const int tilesM = (t.M + BM - 1) / BM, tilesN = (t.N + BN - 1) / BN;
    if ((int)blockIdx.x >= tilesM * tilesN) return;
    // the tiles of one row block are consecutive CTAs, so that its A rows are fetched from HBM
    // once and read from L2 by the other column tiles (B, one tensor per task, stays in L2)
    const int n0 = (blockIdx.x % tilesN) * BN, m0 = (blockIdx.x / tilesN) * BM;
    constexpr int EK = KBYTES / (KIND == 0 ? 4 : 2);  // elements of K per k-block
    const int nk = (t.K + EK - 1) / EK;
    constexpr uint32_t A_BYTES = BM * KBYTES, B_BYTES = BN * KBYTES;  // one k-block
    // a ring stage holds ksub k-blocks: one full/empty barrier round trip per stage (two
    // halve the round trips, one keeps rings small enough for two CTAs per SM)
    const uint32_t A_STAGE = A_BYTES * ksub, B_STAGE = B_BYTES * ksub;
    const int nst = (nk + ksub - 1) / ksub;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + stages * A_STAGE;
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accum;
    __shared__ uint32_t tmem_base;
    __shared__ int issued;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accum, 1);
        issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&gt->map_a);
        prefetch_map(&gt->map_b);
    }
    if (warp == 0) tmem_alloc(&tmem_base, BN < 32 ? 32 : BN);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    // Everything above reads only the static task descriptor, so it may overlap the previous
    // kernel (programmatic dependent launch); the active flag and the operands are its output.
    grid_dependency_wait();
    if (t.active && *t.active == 0) {
        if (warp == 0) tmem_dealloc(tmem, BN < 32 ? 32 : BN);
        return;
    }

    if (warp == 0 && lane == 0) {
        // TMA producer: stage ks holds k-blocks ks*ksub .. (the last stage may hold fewer)
        for (int ks = 0; ks < (stall ? 0 : nst); ++ks) {
            const int s = ks % stages, r = ks / stages;
            if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1, err)) break;
            const int na = min(ksub, nk - ks * ksub);
            mbar_expect_tx(&full[s], (uint32_t)na * (A_BYTES + B_BYTES));
            for (int a = 0; a < na; ++a) {
                const int kb = ks * ksub + a;
                tma_load_2d(sA + s * A_STAGE + a * A_BYTES, &gt->map_a, &full[s], kb * EK, m0);
                tma_load_2d(sB + s * B_STAGE + a * B_BYTES, &gt->map_b, &full[s], kb * EK, n0);
            }
            issued = ks + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t ID = idesc(KIND, BN);
        bool ok = true;
        for (int ks = 0; ks < nst && ok; ++ks) {
            const int s = ks % stages, r = ks / stages;
            ok = mbar_wait(&full[s], r & 1, err);
            if (!ok) break;
            fence_after();
            const int na = min(ksub, nk - ks * ksub);
            for (int a = 0; a < na; ++a) {
                const int kb = ks * ksub + a;
                const uint32_t a0 = smem_u32(sA + s * A_STAGE + a * A_BYTES), b0 = smem_u32(sB + s * B_STAGE + a * B_BYTES);
#pragma unroll
                for (int k = 0; k < KBYTES / 32; ++k)  // 32 bytes of K per instruction, K order as in one stage per k-block
                    umma<KIND>(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), ID, (kb | k) ? 1u : 0u);
            }
            umma_commit(&empty[s]);
        }
        umma_commit(&accum);
    }
    __syncwarp();
    // epilogue: every warp waits for the accumulator, stages its 32 rows in shared memory
    // (the operand ring is free: every issued copy was consumed by a finished MMA)
    const bool ready = mbar_wait(&accum, 0, err);
    launch_dependents();  // the next kernel may start its prologue during this epilogue
    fence_after();
    const int all_ready = __syncthreads_and(ready ? 1 : 0);
    if (all_ready) {
        const int ncols = min(BN, t.N - n0), rows = min(BM, t.M - m0);
        float* tile = (float*)smem;
        long long* roff = (long long*)(tile + BM * (EC + 1));
        long long* coff = roff + BM;
        const int row = warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < ncols; c0 += EC) {
            const int cn = min(EC, ncols - c0);
            const int nchunk = (cn + 15) & ~15;  // tcgen05.ld is warp-collective: uniform bound
            __syncthreads();                     // the previous chunk has been written out
#pragma unroll 1
            for (int c = 0; c < nchunk; c += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + c), v);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c + j < EC) tile[row * (EC + 1) + c + j] = __uint_as_float(v[j]);
            }
            for (int dst = 0; dst < (t.C2 ? 2 : 1); ++dst) {
                void* out = dst ? t.C2 : t.C;
                const long long sm1 = dst ? t.d_m1 : t.c_m1, sm2 = dst ? t.d_m2 : t.c_m2;
                const long long sn1 = dst ? t.d_n1 : t.c_n1, sn2 = dst ? t.d_n2 : t.c_n2;
                const int x3 = (t.x3 >> (2 * dst)) & 3;
                epilogue_dest(tile, roff, coff, rows, cn, m0, n0 + c0, t.M2, t.N2, sm1, sm2, sn1, sn2, t.out_kind,
                              t.alpha, out, x3, dst ? t.kseg2 : t.kseg);
            }
        }
    }
    fence_before();
    __syncthreads();
    // drain: the MMAs issued must have finished before TMEM is released, and the producer's
    // copies must have landed before shared memory is.  On success the MMA warp already waited
    // for every issued copy and the epilogue for every MMA, so only a pipeline that stopped on
    // a timed-out wait (here or in another CTA) can still have work in flight.  The MMA warp
    // commits the accumulator barrier after its loop in every case, so it completes once the
    // MMAs issued before it have; these waits ignore the error word.
    if (!all_ready && threadIdx.x == 0) {
        mbar_wait_own(&accum, 0);
        const int n_issued = issued;
        for (int kb = (n_issued > stages ? n_issued - stages : 0); kb < n_issued; ++kb)
            mbar_wait_own(&full[kb % stages], (kb / stages) & 1);
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BN < 32 ? 32 : BN);
}

}  // namespace tc

// Dynamic shared memory: the operand ring, or the staged epilogue tile and its offsets
// if that is larger, plus 1 KB for the 1024-byte alignment of the swizzled ring.
static size_t tc_smem(int stages, int bn, int ksub) {
    const size_t ring = (size_t)stages * (tc::BM + bn) * tc::KBYTES * ksub;
    const size_t tile = (size_t)tc::BM * (tc::EC + 1) * sizeof(float) + (size_t)(tc::BM + tc::EC) * sizeof(long long);
    return std::max(ring, tile) + 1024;
}

// Deepest ring (stages of ksub k-blocks) that fits the 227 KB of shared memory a CTA may hold
// (2 KB kept for the static barriers and the task): for ksub = 1, 8 stages for BN <= 64, 7 for
// 128, 4 for 256; for ksub = 2, 5 / 4 / 3 / 2 for BN = 32 / 64 / 128 / 256.

// Default ring depth: up to 4 stages within ~96 KB of shared memory (so that two CTAs share an
// SM and one's epilogue overlaps the other's loads and MMAs), at least 2, at most the stages
// the K extent needs.
int tc_default_stages(int bn, int kblocks) {  // one k-block per stage
    const int per = (tc::BM + bn) * tc::KBYTES;
    const int depth = std::max(2, std::min(4, (96 * 1024) / per));
    return std::max(1, std::min(std::min(kblocks, depth), tc_max_stages(bn, 1)));
}
int tc_max_stages(int bn, int ksub) {
    if (ksub < 1 || ksub > tc::KSUB_MAX) return 0;
    const size_t per = (size_t)(tc::BM + bn) * tc::KBYTES * ksub;
    const size_t cap = 232448 - 2048 - 1024;
    return std::max(1, std::min(tc::STAGES, (int)(cap / per)));
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
    dim3 grid(max_tiles, ntasks);
    // programmatic dependent launch: the kernel waits (griddepcontrol.wait) before it reads
    // anything an earlier kernel wrote
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define TC_CASE(K_, N_)                                                              \
    if (kind == K_ && bn == N_) return cudaLaunchKernelEx(&cfg, tc::k_tc_gemm<K_, N_>, d_tasks, err, stages, ksub, stall);
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
