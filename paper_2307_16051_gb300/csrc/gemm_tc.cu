// gemm_tc.cu — trailing update of the half-precision LU on the 5th-generation
// tensor cores:  C <- fl16(C - A Bt^T), A = L21 (M x K), Bt = U12^T (Nc x K),
// binary16 operands, binary32 accumulation in tensor memory (Section 2: the
// factorisation of J_h in half precision; the update is its O(N^3) part).
//
// One CTA per 128 x 128 output tile, 128 threads:
//   * thread 0 loads all K/64 operand slabs of the tile with TMA (128-byte
//     swizzle, one mbarrier with a transaction count), then issues K/16
//     tcgen05.mma (kind::f16, M=128, N=128, K=16) into a 128-column TMEM
//     accumulator and commits them to a second mbarrier;
//   * all four warps read their 32 TMEM lanes (tcgen05.ld 32x32b) and apply
//     C = fl16(C - acc) in the epilogue.
// K <= 256, so the whole K extent is staged at once (the persistent kernel
// below streams any K).
// Each wait is bounded; on timeout the CTA records the error, waits (again
// bounded) for its own copies, releases its tensor memory and returns.
// No cluster multicast: every CTA loads its own tiles.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace nl {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 64;
constexpr int kTcThreads = 128;
constexpr long long kTcWaitCycles = 2000000000LL;

__host__ __device__ constexpr uint32_t tc_idesc() { return tc_idesc_mn(kTcBM, kTcBN); }

// One 128 x 128 output tile at (m0, n0) of C (M x Nc).  The A slab kt of the
// tile is the TMA box at (ax + 64 kt, ay + m0) of tmA, the B slab the box at
// (64 kt, n0) of tmB.  tmA / tmB: generic addresses of the tensor maps (kernel
// parameter or global memory).
__device__ __forceinline__ void tc_gemm_tile(const CUtensorMap* tmA, const CUtensorMap* tmB, int ax, int ay, int M,
                                             int Nc, int K, __half* __restrict__ C, int64_t ldc, int m0, int n0,
                                             unsigned* __restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* basep = smem_raw + (base - raw);
    const int KT = K / kTcBK;
    const uint32_t a_sz = kTcBM * 128, b_sz = kTcBN * 128;  // bytes per 64-wide slab
    const uint32_t sA = base, sB = base + KT * a_sz;
    uint64_t* bars = reinterpret_cast<uint64_t*>(basep + KT * (a_sz + b_sz));
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    const uint32_t bar_load = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int failed;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)kTcBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_load));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)KT * (a_sz + b_sz);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_load), "r"(bytes) : "memory");
        for (int kt = 0; kt < KT; ++kt) {
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                    sA + kt * a_sz),
                "l"(tmA), "r"(ax + kt * kTcBK), "r"(ay + m0), "r"(bar_load)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                    sB + kt * b_sz),
                "l"(tmB), "r"(kt * kTcBK), "r"(n0), "r"(bar_load)
                : "memory");
        }
        if (!mbar_wait(bar_load, 0, kTcWaitCycles)) {
            atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
            failed = 1;
            mbar_wait(bar_load, 0, kTcWaitCycles);  // let copies in flight land
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = tc_idesc();
            for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
                for (int kk = 0; kk < kTcBK / 16; ++kk) {
                    uint64_t ad = sw128_desc(sA + kt * a_sz + kk * 32);
                    uint64_t bd = sw128_desc(sB + kt * b_sz + kk * 32);
                    uint32_t acc = (kt | kk) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                         : "memory");
        }
    }
    // The epilogue's C tile does not depend on the MMAs: load it now so its
    // latency overlaps them (each thread: its row, 128 columns, 16 x 16 B).
    const int row = m0 + warp * 32 + lane;
    __half* Crow = C + (int64_t)min(row, M - 1) * ldc;
    const bool full = (row < M) && (n0 + kTcBN <= Nc);
    uint4 cpre[kTcBN / 8];
    if (full) {
        const uint4* p = reinterpret_cast<const uint4*>(Crow + n0);
#pragma unroll
        for (int q = 0; q < kTcBN / 8; ++q) cpre[q] = p[q];
    }
    __syncthreads();
    bool ok = !failed;
    if (ok && !mbar_wait(bar_mma, 0, kTcWaitCycles)) {
        atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
        mbar_wait(bar_mma, 0, kTcWaitCycles);  // let the MMAs in flight finish
        ok = false;
    }
    ok = !__syncthreads_or(!ok);  // warp-uniform: the TMEM loads below are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
#pragma unroll
        for (int c = 0; c < kTcBN; c += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int col0 = n0 + c;
            if (full) {
                uint4* p = reinterpret_cast<uint4*>(Crow + col0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 v = cpre[c / 8 + q];
                    uint32_t wds[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __half2 h2;
                        memcpy(&h2, &wds[e], 4);
                        float2 f = __half22float2(h2);
                        f.x -= __uint_as_float(r[q * 8 + 2 * e]);
                        f.y -= __uint_as_float(r[q * 8 + 2 * e + 1]);
                        h2 = __floats2half2_rn(f.x, f.y);
                        memcpy(&wds[e], &h2, 4);
                    }
                    p[q] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                }
            } else if (row < M) {
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (col0 + e < Nc)
                        Crow[col0 + e] = __float2half_rn(__half2float(Crow[col0 + e]) - __uint_as_float(r[e]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTcBN));
    }
}

__global__ void __launch_bounds__(kTcThreads) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB, int M, int Nc,
                                                        int K, __half* __restrict__ C, int64_t ldc,
                                                        unsigned* __restrict__ err, const int* __restrict__ flag)
{
    if (flag && *(volatile const int*)flag) return;  // the LU's fast path was abandoned
    tc_gemm_tile(&tmA, &tmB, 0, 0, M, Nc, K, C, ldc, (int)blockIdx.y * kTcBM, (int)blockIdx.x * kTcBN, err);
}

// ------------------------------------------------ persistent, pipelined --
// The same update C <- fl16(C - A Bt^T) with one CTA per SM looping over the
// output tiles (tile = blockIdx.x + i * gridDim.x) and four warp roles, each
// stage of work double-buffered:
//   warp 0 (one thread): TMA loads of the A and B slabs of tile i into the
//     operand ring's slots as the MMAs free them;
//   warp 1 (one thread): K/16 tcgen05.mma into TMEM accumulator i % 2 (BN
//     columns each) once the epilogue has read tile i-2's accumulator, then
//     tcgen05.commit to "accumulator full" and to "operand stage free";
//   warps 2-5: epilogue.  Each thread owns one tile row (its warp's TMEM
//     lane quarter): tcgen05.ld of the accumulator row (then "accumulator
//     free"), C from C buffer i % kPCBuf (128-byte swizzle), fl16(C - acc)
//     written back in place, a proxy fence and an arrival on "C written";
//   warp 6 (one thread): the C tiles' traffic.  TMA load of C for tile i
//     into buffer i % kPCBuf, and for each finished tile the TMA bulk store of
//     its C buffer, whose completed read of the buffer frees it for tile
//     i + kPCBuf.
// Loads, MMAs, epilogue and stores of consecutive tiles overlap, and all
// global traffic is TMA (coalesced, asynchronous).  Per element the
// arithmetic is the per-tile kernel's: the same K/16 MMAs in the same order,
// then one subtraction and one rounding.  Tiles are 128 x BN (BN = 128, or
// 256 for deep updates: one N = 256 MMA per 16 of K).  The operands stream
// through a ring of kPRing slots of one 64-wide K slab of A and of B each
// (16 KB + BN x 128 B), so K is any multiple of 64 up to kPMaxK: C stays in
// the tensor-memory accumulator for the whole K extent and is read and
// written once per update, whatever K (the LU's outer block).  With two or
// more C buffers one C tile is in flight to or from memory while the epilogue
// works on another.  Every wait is bounded; a timeout marks the CTA aborted,
// every role leaves its loop, in-flight copies and MMAs are waited for
// (bounded), and tensor memory is released.
constexpr int kPThreads = 224;
constexpr uint32_t kPSlab = 128 * 128;  // bytes of one 128-row x 64-column binary16 slab
// Ring shapes (operand slots, C buffers) of the 128 x 128 form, 225 KB of shared
// memory either way.  Deep updates (K = 256; from K = 512 the wide form below)
// stream many operand slabs per C tile and are bound by
// the operand bytes in flight against the L2 latency (ncu, N = 8192, K = 512,
// four slots: L2 43%, DRAM 36%, tensor pipe 35%), so they take five slots and
// two C buffers; shallow ones (K <= 128, and the grouped update) move more C
// than operands and keep three C buffers.  Measured on GB300: the N = 32768
// factorisation's K = 512 updates 25.4 ms with (5, 2) against 27.8 with (4, 3)
// and 28.3 with (6, 1); the batch's K = 64 grouped updates 4% faster with (4, 3).
constexpr int kPRingDeep = 5, kPCBufDeep = 2;
constexpr int kPRingShallow = 4, kPCBufShallow = 3;
constexpr int kPMaxK = 1024;               // largest K of one update
// Updates with K >= 512 take 128 x 256 tiles (one M = 128, N = 256 MMA per 16 of K, the two
// accumulators in all 512 tensor-memory columns): a quarter fewer operand bytes per flop than
// 128 x 128, in three operand slots (48 KB each) and one 64 KB C buffer.  Bitwise the same
// results.  Measured on GB300, the N = 32768 factorisation's K = 512 updates: 23.7 ms against
// 25.4 with 128 x 128 tiles (two slots and two C buffers: 28.8 ms); at K = 256 the single C
// buffer serialises the C traffic (50.4 against 35.8 ms), so shallower updates keep 128 x 128.
constexpr int kTcBNWide = 256, kPRingWide = 3, kPCBufWide = 1;

static size_t p_smem_bytes(int ring, int cbuf, int bn = kTcBN)
{
    return 1024 + (size_t)ring * (kPSlab + (size_t)bn * 128) + (size_t)cbuf * bn * 256 + 256;
}

// Where tile `it` of a persistent CTA reads and writes: the A slabs at
// (ax + 64 kt, ay) of map a, the B slabs at (64 kt, by) of map b, the C tile's
// two boxes at (cx + 64 j, cy) of map c; `store` is false for a matrix whose
// factorisation has been abandoned (its tile is computed but not written).
struct TileRef {
    const CUtensorMap *a, *b, *c;
    int ax, ay, by, cx, cy;
    bool store;
};

// Single update: the maps are kernel parameters (tmA, tmB, tmC), tiles in
// row-major order over the M x Nc output; with cross set only the first tile
// column (every tile row) and the rest of the first tile row, the part of the
// trailing matrix the next panel of an LU reads.  Grouped update: task t of the
// step's list is {instance, m0, n0} of that instance's A22 (rows and columns
// from K + w), read through the instance's whole-matrix map (A and C) and
// its U12^T map (B); rows and columns past the instance's N read as zero and
// are not stored.
template <bool GROUPED, int kPRing, int kPCBuf, int BN = kTcBN>
__device__ __forceinline__ void tc_gemm_persistent(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                                   const CUtensorMap* tmC, int M, int Nc, int K,
                                                   const GInst* __restrict__ ginst, const TmapBytes* __restrict__ gmaps,
                                                   const GTask* __restrict__ gtasks, int ntasks, int gK, int gw,
                                                   unsigned* __restrict__ err, int cross = 0)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* basep = smem_raw + (base - raw);
    const int KT = K / kTcBK;
    constexpr uint32_t kSlot = kPSlab + (uint32_t)BN * 128;  // one A slab and one B slab
    constexpr uint32_t kCB = (uint32_t)BN * 256;               // one C tile: BN / 64 boxes
    const uint32_t ring_bytes = (uint32_t)kPRing * kSlot;
    const uint32_t sAB = base, sCb = base + ring_bytes;  // operand slots, then C buffers
    uint64_t* bars = reinterpret_cast<uint64_t*>(basep + ring_bytes + kPCBuf * kCB);
    // bars: slot_full[4] (0..3), slot_empty[4] (4..7), tfull[2] (8, 9), tempty[2] (10, 11),
    // c_full[3] (12..14), c_done[3] (15..17); then the TMEM address
    constexpr int bFULL = 0, bEMPTY = kPRing, bTFULL = 2 * kPRing, bTEMPTY = 2 * kPRing + 2,
                  bCFULL = 2 * kPRing + 4, bCDONE = 2 * kPRing + 4 + kPCBuf;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + bCDONE + kPCBuf);
    __shared__ int aborted;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (Nc + BN - 1) / BN, tiles_m = (M + kTcBM - 1) / kTcBM;
    const int ntiles = GROUPED ? ntasks : (cross ? tiles_m + tiles_n - 1 : tiles_n * tiles_m);
    const int nmine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto bar = [&](int k) { return smem_u32(&bars[k]); };
    auto fail = [&]() {
        atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
        *(volatile int*)&aborted = 1;
    };
    auto ref = [&](int it) {
        const int tile = blockIdx.x + it * gridDim.x;
        TileRef r;
        if constexpr (GROUPED) {
            const GTask t = gtasks[tile];
            r.a = r.c = reinterpret_cast<const CUtensorMap*>(&gmaps[2 * t.inst]);
            r.b = reinterpret_cast<const CUtensorMap*>(&gmaps[2 * t.inst + 1]);
            r.ax = gK;
            r.ay = r.cy = gK + gw + t.a;
            r.by = t.b;
            r.cx = gK + gw + t.b;
            r.store = *(volatile const int*)ginst[t.inst].flag == 0;
        } else {
            int m0, n0;
            if (cross) {  // tiles (i, 0) for every i, then (0, j) for j >= 1
                m0 = tile < tiles_m ? tile * kTcBM : 0;
                n0 = tile < tiles_m ? 0 : (tile - tiles_m + 1) * BN;
            } else {
                m0 = (tile / tiles_n) * kTcBM;
                n0 = (tile % tiles_n) * BN;
            }
            r.a = tmA;
            r.b = tmB;
            r.c = tmC;
            r.ax = 0;
            r.ay = r.cy = m0;
            r.by = n0;
            r.cx = n0;
            r.store = true;
        }
        return r;
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2u * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        aborted = 0;
        for (int k = 0; k < kPRing; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(bFULL + k)));     // slot full (TMA)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(bEMPTY + k)));    // slot free (MMA commit)
        }
        for (int k = 0; k < 2; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(bTFULL + k)));    // tfull (MMA commit)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(bar(bTEMPTY + k))); // tempty (epilogue)
        }
        for (int k = 0; k < kPCBuf; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(bCFULL + k)));    // c_full (TMA)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(bar(bCDONE + k)));  // c_done (epilogue)
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: slab g (tile it, K slab kt; g = it KT + kt) into slot g % kPRing once the
            // MMAs of slab g - kPRing are done with it
            long long g = 0;
            bool ok = true;
            for (int it = 0; it < nmine && ok && !*(volatile int*)&aborted; ++it) {
                const TileRef r = ref(it);
                for (int kt = 0; kt < KT; ++kt, ++g) {
                    const int s = (int)(g % kPRing);
                    const uint32_t ph = (uint32_t)(g / kPRing) & 1u;
                    if (g >= kPRing && !mbar_wait(bar(bEMPTY + s), ph ^ 1u, kTcWaitCycles)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint32_t sA = sAB + (uint32_t)s * kSlot, sB = sA + kPSlab;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(bFULL + s)),
                                 "r"(kSlot)
                                 : "memory");
                    tma_load_2d(sA, r.a, r.ax + kt * kTcBK, r.ay, bar(bFULL + s));
                    tma_load_2d(sB, r.b, kt * kTcBK, r.by, bar(bFULL + s));
                }
            }
            // copies in flight land before the CTA's shared memory goes away
            for (long long j = (g >= kPRing ? g - kPRing : 0); j < g; ++j)
                mbar_wait(bar(bFULL + (int)(j % kPRing)), (uint32_t)(j / kPRing) & 1u, kTcWaitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile it accumulates its KT slabs into accumulator it % 2, each slab's
            // MMAs committed to its slot's "free" barrier, the tile's to "accumulator full"
            const uint32_t idesc = tc_idesc_mn(kTcBM, BN);
            long long g = 0;
            bool ok = true;
            for (int it = 0; it < nmine && ok && !*(volatile int*)&aborted; ++it) {
                const int b = it & 1;
                const uint32_t pht = (uint32_t)(it >> 1) & 1u;
                if (it >= 2 && !mbar_wait(bar(bTEMPTY + b), pht ^ 1u, kTcWaitCycles)) {
                    fail();
                    break;
                }
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int kt = 0; kt < KT; ++kt, ++g) {
                    const int s = (int)(g % kPRing);
                    const uint32_t ph = (uint32_t)(g / kPRing) & 1u;
                    if (!mbar_wait(bar(bFULL + s), ph, kTcWaitCycles)) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sA = sAB + (uint32_t)s * kSlot, sB = sA + kPSlab;
#pragma unroll
                    for (int kk = 0; kk < kTcBK / 16; ++kk) {
                        const uint64_t ad = sw128_desc(sA + kk * 32);
                        const uint64_t bd = sw128_desc(sB + kk * 32);
                        const uint32_t acc = (kt | kk) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     bar(bEMPTY + s))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 bar(bTFULL + b))
                             : "memory");
            }
            // every issued MMA is complete (the last commit covers all earlier ones) before
            // tensor memory is released
            if (g > 0)
                mbar_wait(bar(bEMPTY + (int)((g - 1) % kPRing)), (uint32_t)((g - 1) / kPRing) & 1u, kTcWaitCycles);
        }
    } else if (warp == 6) {
        if (lane == 0) {
            // C traffic: loads for tiles 0..2, then per finished tile i its store
            // and, once the store has read the buffer, the load for tile i + kPCBuf
            int loaded = 0;
            for (int it = 0; it < kPCBuf && it < nmine; ++it) {
                const TileRef r = ref(it);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(bCFULL + it)),
                             "r"(kCB)
                             : "memory");
                for (int j = 0; j < BN / 64; ++j)
                    tma_load_2d(sCb + it * kCB + j * kPSlab, r.c, r.cx + j * kTcBK, r.cy, bar(bCFULL + it));
                loaded = it + 1;
            }
            for (int it = 0; it < nmine && !*(volatile int*)&aborted; ++it) {
                const int s = it % kPCBuf;
                const uint32_t ph = (uint32_t)(it / kPCBuf) & 1u;
                if (!mbar_wait(bar(bCDONE + s), ph, kTcWaitCycles)) {
                    fail();
                    break;
                }
                const TileRef r = ref(it);
                if (r.store)
                    for (int j = 0; j < BN / 64; ++j)
                        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                                         r.c),
                                     "r"(r.cx + j * kTcBK), "r"(r.cy), "r"(sCb + s * kCB + j * kPSlab)
                                     : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                if (it + kPCBuf < nmine) {
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    const TileRef rn = ref(it + kPCBuf);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(bCFULL + s)),
                                 "r"(kCB)
                                 : "memory");
                    for (int j = 0; j < BN / 64; ++j)
                        tma_load_2d(sCb + s * kCB + j * kPSlab, rn.c, rn.cx + j * kTcBK, rn.cy, bar(bCFULL + s));
                    loaded = it + kPCBuf + 1;
                }
            }
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
            if (*(volatile int*)&aborted)
                for (int it = (loaded >= kPCBuf ? loaded - kPCBuf : 0); it < loaded; ++it)
                    mbar_wait(bar(bCFULL + it % kPCBuf), (uint32_t)(it / kPCBuf) & 1u, kTcWaitCycles);
        }
    } else {
        const int q = warp & 3;       // TMEM lane quarter of this warp (warps 2..5 -> 2, 3, 0, 1)
        const int r = q * 32 + lane;  // tile row of this thread
        const uint32_t swz = (uint32_t)(r & 7);
        for (int it = 0; it < nmine; ++it) {
            const int s = it % kPCBuf, b = it & 1;
            const uint32_t ph = (uint32_t)(it >> 1) & 1u, phc = (uint32_t)(it / kPCBuf) & 1u;
            const bool ok = !*(volatile int*)&aborted && mbar_wait(bar(bTFULL + b), ph, kTcWaitCycles) &&
                            mbar_wait(bar(bCFULL + s), phc, kTcWaitCycles);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t* cst = basep + ring_bytes + s * kCB;  // C buffer it % kPCBuf
#pragma unroll
            for (int c = 0; c < BN; c += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (c + 32 == BN) {
                    // the whole accumulator row is in registers: the buffer may be reused
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(bar(bTEMPTY + b));
                }
                // columns c .. c+31: box c / 64, 16-byte chunks (c % 64) / 8 .. + 3, swizzled by row
                uint8_t* rowp = cst + (c / 64) * kPSlab + r * 128;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const uint32_t chunk = (uint32_t)((c % 64) / 8 + h) ^ swz;
                    uint4* p = reinterpret_cast<uint4*>(rowp + chunk * 16);
                    const uint4 x = *p;
                    uint32_t wds[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __half2 h2;
                        memcpy(&h2, &wds[e], 4);
                        float2 f = __half22float2(h2);
                        f.x -= __uint_as_float(v[h * 8 + 2 * e]);
                        f.y -= __uint_as_float(v[h * 8 + 2 * e + 1]);
                        h2 = __floats2half2_rn(f.x, f.y);
                        memcpy(&wds[e], &h2, 4);
                    }
                    *p = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                }
            }
            // this row of the tile is written: visible to the TMA store, then signalled
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(bar(bCDONE + s));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * BN));
    }
}

template <int RING, int CBUF, int BN = kTcBN>
__global__ void __launch_bounds__(kPThreads, 1) k_tc_gemm_p(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB,
                                                            const __grid_constant__ CUtensorMap tmC, int M, int Nc,
                                                            int K, unsigned* __restrict__ err,
                                                            const int* __restrict__ flag, int cross)
{
    if (flag && *(volatile const int*)flag) return;  // the LU's fast path was abandoned
    tc_gemm_persistent<false, RING, CBUF, BN>(&tmA, &tmB, &tmC, M, Nc, K, nullptr, nullptr, nullptr, 0, 0, 0, err,
                                              cross);
}

__global__ void __launch_bounds__(kPThreads, 1) k_tc_gemm_pg(const GInst* __restrict__ inst,
                                                             const TmapBytes* __restrict__ maps,
                                                             const GTask* __restrict__ tasks, int ntasks, int K, int w,
                                                             unsigned* __restrict__ err)
{
    tc_gemm_persistent<true, kPRingShallow, kPCBufShallow>(nullptr, nullptr, nullptr, 0, 0, w, inst, maps, tasks, ntasks,
                                                           K, w, err);
}

// Grouped trailing update of outer step [K, K + w) of many matrices: task
// {inst, m0, n0} updates tile (m0, n0) of instance inst's A22 (rows and
// columns from K + w) with L21 (rows from K + w, columns K .. K + w) read
// through the instance's whole-matrix tensor map and U12^T through its
// buffer's map.  Rows past N read as zero (TMA fill) and are not stored.
__global__ void __launch_bounds__(kTcThreads) k_tc_gemm_g(const GInst* __restrict__ inst,
                                                          const TmapBytes* __restrict__ maps,
                                                          const GTask* __restrict__ tasks, int K, int w,
                                                          unsigned* __restrict__ err)
{
    const GTask t = tasks[blockIdx.x];
    const GInst I = inst[t.inst];
    if (*(volatile const int*)I.flag) return;
    const int rest = I.N - K - w;
    __half* A = reinterpret_cast<__half*>(I.A);
    tc_gemm_tile(reinterpret_cast<const CUtensorMap*>(&maps[2 * t.inst]),
                 reinterpret_cast<const CUtensorMap*>(&maps[2 * t.inst + 1]), K, K + w, rest, rest, w,
                 A + (int64_t)(K + w) * I.ld + K + w, I.ld, t.a, t.b, err);
}

// ------------------------------------------------------------------- host --

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static int g_tc_state = -1;  // -1 unknown, 0 unsupported, 1 supported
static unsigned* g_tc_err = nullptr;

bool tc_gemm_supported()
{
    if (g_tc_state >= 0) return g_tc_state == 1;
    g_tc_state = 0;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10) return false;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    if (cudaMalloc((void**)&g_tc_err, sizeof(unsigned)) != cudaSuccess) return false;
    cudaMemset(g_tc_err, 0, sizeof(unsigned));
    if (set_max_dynamic_smem((const void*)k_tc_gemm) != NL_OK) return false;
    if (set_max_dynamic_smem((const void*)k_tc_gemm_g) != NL_OK) return false;
    if (set_max_dynamic_smem((const void*)k_tc_gemm_p<kPRingDeep, kPCBufDeep>) != NL_OK) return false;
    if (set_max_dynamic_smem((const void*)k_tc_gemm_p<kPRingShallow, kPCBufShallow>) != NL_OK) return false;
    if (set_max_dynamic_smem((const void*)k_tc_gemm_p<kPRingWide, kPCBufWide, kTcBNWide>) != NL_OK) return false;
    if (set_max_dynamic_smem((const void*)k_tc_gemm_pg) != NL_OK) return false;
    g_tc_state = 1;
    return true;
}

static size_t tc_smem_bytes(int K)
{
    const int KT = K / kTcBK;
    // at least 58 KB so that at most three CTAs (3 x 128 TMEM columns) share an SM
    return std::max<size_t>(1024 + (size_t)KT * (kTcBM + kTcBN) * 128 + 64, 58 * 1024);
}

static bool encode_2d(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                      uint32_t box_inner, uint32_t box_outer)
{
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld_elems * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

nl_status tc_gemm16_update(int M, int Nc, int K, const __half* A, int64_t lda, const __half* Bt, int64_t ldbt,
                           __half* C, int64_t ldc, cudaStream_t st, const int* flag, bool per_tile, bool cross,
                           int max_ctas)
{
    if (M <= 0 || Nc <= 0) return NL_OK;
    if (!tc_gemm_supported()) {
        set_error("tcgen05 GEMM: needs an sm_100-family device and the tensor-map driver entry point");
        return NL_ECUDA;
    }
    if (K % kTcBK || K < kTcBK || K > kPMaxK || (per_tile && K > 256) || (lda % 8) || (ldbt % 8) || (ldc % 8) ||
        ((uintptr_t)A & 15) || ((uintptr_t)Bt & 15) || ((uintptr_t)C & 15)) {
        set_error("tcgen05 GEMM: K must be a multiple of 64 (<= 1024; <= 256 one tile per CTA), leading dimensions "
                  "multiples of 8, pointers 16-byte aligned");
        return NL_EINVAL;
    }
    const bool wide = !per_tile && !cross && K >= 512;
    const int bn = wide ? kTcBNWide : kTcBN;
    CUtensorMap tmA, tmB;
    if (!encode_2d(&tmA, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, kTcBK, kTcBM) ||
        !encode_2d(&tmB, Bt, (uint64_t)K, (uint64_t)Nc, (uint64_t)ldbt, kTcBK, (uint32_t)bn)) {
        set_error("tcgen05 GEMM: cuTensorMapEncodeTiled failed");
        return NL_ECUDA;
    }
    if (!per_tile) {
        // persistent pipelined kernel: one CTA per SM (at most one per tile)
        CUtensorMap tmC;
        if (!encode_2d(&tmC, C, (uint64_t)Nc, (uint64_t)M, (uint64_t)ldc, kTcBK, kTcBM)) {
            set_error("tcgen05 GEMM: cuTensorMapEncodeTiled failed (C)");
            return NL_ECUDA;
        }
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (nsm < 1) nsm = 1;
        }
        const long long ntiles = cross ? (long long)cdiv(Nc, kTcBN) + cdiv(M, kTcBM) - 1
                                       : (long long)cdiv(Nc, bn) * cdiv(M, kTcBM);
        // A small shallow update (K <= 128, at most 8 tiles per SM: a one-level panel's at
        // N <= ~4600) is short and bound by its C traffic; half the SMs leave the other half
        // to concurrent solves' latency-bound panels (the sweep of five concurrent solves at
        // N = 4096 measured 123 against 119 solves/s with every SM, 120 with a third; one
        // solve alone is 2% slower).  Larger and deep updates take every SM (capped, the
        // N = 32768 factorisation with nb = 128 took 104 instead of 82 ms).
        // (The cross of a look-ahead LU is on its critical path: a tile per CTA where it can.)
        const bool small = !cross && K < 256 && ntiles <= 8LL * nsm;
        unsigned grid = (unsigned)std::min<long long>(ntiles, small ? std::max(1, nsm / 2) : nsm);
        if (small && max_ctas > 0) grid = std::min<unsigned>(grid, (unsigned)max_ctas);
        const char* cls = cross ? "k_tc_gemm_x" : "k_tc_gemm";
        prof_begin(cls, st);
        if (wide)
            k_tc_gemm_p<kPRingWide, kPCBufWide, kTcBNWide>
                <<<grid, kPThreads, p_smem_bytes(kPRingWide, kPCBufWide, kTcBNWide), st>>>(tmA, tmB, tmC, M, Nc, K,
                                                                                         g_tc_err, flag, 0);
        else if (K >= 256)
            k_tc_gemm_p<kPRingDeep, kPCBufDeep><<<grid, kPThreads, p_smem_bytes(kPRingDeep, kPCBufDeep), st>>>(
                tmA, tmB, tmC, M, Nc, K, g_tc_err, flag, cross ? 1 : 0);
        else
            k_tc_gemm_p<kPRingShallow, kPCBufShallow><<<grid, kPThreads, p_smem_bytes(kPRingShallow, kPCBufShallow),
                                                         st>>>(tmA, tmB, tmC, M, Nc, K, g_tc_err, flag, cross ? 1 : 0);
        prof_end(cls, st);
        NL_CUDA_OK(cudaGetLastError());
        return NL_OK;
    }
    const size_t smem = tc_smem_bytes(K);
    dim3 grid((unsigned)cdiv(Nc, kTcBN), (unsigned)cdiv(M, kTcBM));
    prof_begin("k_tc_gemm", st);
    k_tc_gemm<<<grid, kTcThreads, smem, st>>>(tmA, tmB, M, Nc, K, C, ldc, g_tc_err, flag);
    prof_end("k_tc_gemm", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

bool tc_encode_instance_maps(const __half* A, int N, int64_t ld, const __half* ut, int nb, TmapBytes* out2)
{
    static_assert(sizeof(TmapBytes) == sizeof(CUtensorMap), "tensor-map size");
    if (!tc_gemm_supported()) return false;
    return encode_2d(reinterpret_cast<CUtensorMap*>(&out2[0]), A, (uint64_t)N, (uint64_t)N, (uint64_t)ld, kTcBK,
                     kTcBM) &&
           encode_2d(reinterpret_cast<CUtensorMap*>(&out2[1]), ut, (uint64_t)nb, (uint64_t)round_up(N, 128),
                     (uint64_t)nb, kTcBK, kTcBN);
}

// ------------------------------------------ single-precision C update --
// C <- C - A B for binary32 C and binary32 operands whose values are binary16
// numbers (the two-level LU's inner updates on its single-precision shadow:
// multipliers and U entries are rounded to binary16 when they are formed),
// K <= 128.  One CTA of 256 threads per 128 x 128 tile: the threads convert
// the operands to binary16 (exact) into 128-byte-swizzled K-major slabs (the
// layout a TMA load with 128-byte swizzle writes: 16-byte chunk c of row r at
// (r / 8) * 1024 + (r % 8) * 128 + ((c ^ (r % 8)) * 16)), zero beyond M, N and
// K; thread 0 issues the ceil(K / 16) tcgen05.mma of kind::f16 into a
// 128-column TMEM accumulator; each thread then applies C = C - acc to 64
// entries of one row (its C segment loaded while the MMAs run).  Per entry the K products are summed by the tensor cores and applied
// with one binary32 rounding (the SIMT update rounds after each product), the
// tensor-core update's rounding.  The wait is bounded; on timeout the CTA
// records the error, waits (bounded) for its MMAs, skips the update, and
// releases its tensor memory.
constexpr int kUfThreads = 256;
constexpr uint32_t kUfSlab = 128 * 128;  // bytes: 128 rows x 64 binary16
static size_t uf_smem_bytes() { return 1024 + 4 * (size_t)kUfSlab + 64; }

__device__ __forceinline__ uint4 pack8_h(const float* v)
{
    uint4 u;
    __half2 h;
    h = __floats2half2_rn(v[0], v[1]);
    memcpy(&u.x, &h, 4);
    h = __floats2half2_rn(v[2], v[3]);
    memcpy(&u.y, &h, 4);
    h = __floats2half2_rn(v[4], v[5]);
    memcpy(&u.z, &h, 4);
    h = __floats2half2_rn(v[6], v[7]);
    memcpy(&u.w, &h, 4);
    return u;
}

__global__ void __launch_bounds__(kUfThreads) k_tc_update_f32(int M, int Nc, int K, const float* __restrict__ A,
                                                              int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                              float* __restrict__ C, int64_t ldc,
                                                              unsigned* __restrict__ err, const int* __restrict__ flag)
{
    if (flag && *(volatile const int*)flag) return;  // the LU's fast path was abandoned
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* basep = smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + 2 * kUfSlab;
    uint64_t* bars = reinterpret_cast<uint64_t*>(basep + 4 * kUfSlab);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = (int)blockIdx.y * 128, n0 = (int)blockIdx.x * 128;
    const int KT = (K + 63) / 64, nq = 8 * KT;  // slabs and 16-byte chunks per row
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(128u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bool avec = (lda % 4 == 0) && ((((uintptr_t)A) & 15) == 0);
#pragma unroll 4
    for (int idx = tid; idx < 128 * nq; idx += kUfThreads) {
        const int r = idx / nq, q = idx % nq, k0 = 8 * q, i = m0 + r;
        float v[8];
        if (avec && i < M && k0 + 8 <= K) {
            const float4* p = reinterpret_cast<const float4*>(A + (int64_t)i * lda + k0);
            const float4 a = __ldg(p), b = __ldg(p + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (i < M && k0 + e < K) ? __ldg(A + (int64_t)i * lda + k0 + e) : 0.0f;
        }
        // a plain shared store (no asm barrier), so the loads of later chunks can be issued ahead
        *reinterpret_cast<uint4*>(basep + (q >> 3) * kUfSlab + sw128_off(r, q & 7)) = pack8_h(v);
    }
    // B as N x K (K-major): row n holds column n0 + n of B; consecutive threads read consecutive columns
#pragma unroll 4
    for (int idx = tid; idx < 128 * nq; idx += kUfThreads) {
        const int n = idx & 127, q = idx >> 7, k0 = 8 * q, j = n0 + n;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (j < Nc && k0 + e < K) ? __ldg(B + (int64_t)(k0 + e) * ldb + j) : 0.0f;
        *reinterpret_cast<uint4*>(basep + 2 * kUfSlab + (q >> 3) * kUfSlab + sw128_off(n, q & 7)) = pack8_h(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the slabs, for the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot, bar = smem_u32(&bars[0]);
    if (tid == 0) {
        const uint32_t idesc = tc_idesc_mn(128, 128);
        const int ks = (K + 15) / 16;
        for (int s2 = 0; s2 < ks; ++s2) {
            const uint32_t off = (uint32_t)(s2 >> 2) * kUfSlab + (uint32_t)(s2 & 3) * 32;
            const uint64_t ad = sw128_desc(sA + off), bd = sw128_desc(sB + off);
            const uint32_t acc = s2 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
    }
    // warp w: TMEM lanes (rows) 32 (w % 4) .. +31, columns 64 (w / 4) .. +63.  The C
    // segment does not depend on the MMAs: load it while they run.
    const int row = m0 + (warp & 3) * 32 + lane, cbase = (warp >> 2) * 64;
    float* Crow = C + (int64_t)min(row, M - 1) * ldc + n0 + cbase;
    const bool cfull = row < M && n0 + cbase + 64 <= Nc && (ldc % 4 == 0) && ((((uintptr_t)Crow) & 15) == 0);
    float4 cpre[16];
    if (cfull) {
#pragma unroll
        for (int q = 0; q < 16; ++q) cpre[q] = reinterpret_cast<const float4*>(Crow)[q];
    }
    bool ok = mbar_wait(bar, 0, kTcWaitCycles);
    if (!ok) {
        atomicOr(err, (unsigned)ERR_TIMEOUT_OTHER);
        mbar_wait(bar, 0, kTcWaitCycles);  // let the MMAs in flight finish
    }
    ok = !__syncthreads_or(!ok);  // CTA-uniform: the TMEM loads below are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cbase + 32 * h);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (cfull) {
                float4* p4 = reinterpret_cast<float4*>(Crow + 32 * h);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4 x = cpre[8 * h + q];
                    x.x -= __uint_as_float(r[4 * q]);
                    x.y -= __uint_as_float(r[4 * q + 1]);
                    x.z -= __uint_as_float(r[4 * q + 2]);
                    x.w -= __uint_as_float(r[4 * q + 3]);
                    p4[q] = x;
                }
            } else if (row < M) {
                const int j0 = n0 + cbase + 32 * h;
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (j0 + e < Nc) Crow[32 * h + e] -= __uint_as_float(r[e]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
    }
}

nl_status tc_update_f32(int M, int Nc, int K, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                        int64_t ldc, cudaStream_t st, const int* flag)
{
    if (M <= 0 || Nc <= 0 || K <= 0) return NL_OK;
    if (!tc_gemm_supported()) {
        set_error("tcgen05 update: needs an sm_100-family device");
        return NL_ECUDA;
    }
    if (K > 128) {
        set_error("tcgen05 update: K must be at most 128");
        return NL_EINVAL;
    }
    static bool smem_set = false;
    if (!smem_set) {
        if (set_max_dynamic_smem((const void*)k_tc_update_f32) != NL_OK) return NL_ECUDA;
        smem_set = true;
    }
    const dim3 grid((unsigned)cdiv(Nc, 128), (unsigned)cdiv(M, 128));
    prof_begin("k_tc_update32", st);
    k_tc_update_f32<<<grid, kUfThreads, uf_smem_bytes(), st>>>(M, Nc, K, A, lda, B, ldb, C, ldc, g_tc_err, flag);
    prof_end("k_tc_update32", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

nl_status tc_gemm16_grouped(const GInst* inst, const TmapBytes* maps, const GTask* tasks, int ntasks, int K, int w,
                            cudaStream_t st)
{
    if (ntasks <= 0) return NL_OK;
    if (!tc_gemm_supported() || w % kTcBK || w > 256) {
        set_error("grouped tcgen05 GEMM: needs the tensor-core path and a panel width that is a multiple of 64");
        return NL_EINVAL;
    }
    prof_begin("k_tc_gemm", st);
    if (w <= 2 * kTcBK) {
        // persistent: one CTA per SM over the step's task list
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (nsm < 1) nsm = 1;
        }
        const unsigned grid = (unsigned)std::min(ntasks, nsm);
        k_tc_gemm_pg<<<grid, kPThreads, p_smem_bytes(kPRingShallow, kPCBufShallow), st>>>(inst, maps, tasks, ntasks,
                                                                                           K, w, g_tc_err);
    } else {
        k_tc_gemm_g<<<(unsigned)ntasks, kTcThreads, tc_smem_bytes(w), st>>>(inst, maps, tasks, K, w, g_tc_err);
    }
    prof_end("k_tc_gemm", st);
    NL_CUDA_OK(cudaGetLastError());
    return NL_OK;
}

// Device error word of the tensor-core path (read by the solver after a factorisation).
unsigned* tc_error_word() { return g_tc_err; }

}  // namespace nl

extern "C" nl_status nl_k_update32(int64_t M, int64_t Nc, int64_t K, const float* A, int64_t lda, const float* B,
                                   int64_t ldb, float* C, int64_t ldc, void* stream)
{
    using namespace nl;
    set_error("");
    if (M < 0 || Nc < 0 || K < 0 || K > 128 || M > INT32_MAX || Nc > INT32_MAX ||
        (M > 0 && Nc > 0 && K > 0 && (!A || !B || !C || lda < K || ldb < Nc || ldc < Nc))) {
        set_error("nl_k_update32: bad argument (K <= 128, leading dimensions at least the row lengths)");
        return NL_EINVAL;
    }
    return tc_update_f32((int)M, (int)Nc, (int)K, A, lda, B, ldb, C, ldc, (cudaStream_t)stream, nullptr);
}
