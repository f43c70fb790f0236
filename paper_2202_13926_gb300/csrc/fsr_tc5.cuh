// Precision study: the forward 2-D DFT of a block (a3) and the inverse of its
// model (a9) as GEMMs on the fifth-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory), TF32 operands or BF16 hi/lo split products
// (hi.hi + hi.lo + lo.hi), FP32 accumulation; the iteration stays FP32 SIMT.
//
// Both passes of a 2-D DFT are one real GEMM  D (32 x 64) = A (32 x 64) . M
// (64 x 64), A = [Re | Im] of the 32 x 32 complex input (rows m, columns n),
// M = [[Fr, Fi], [-Fi, Fr]], F[n][l] = e^{-j 2 pi n l / 32} (symmetric):
// pass 1 gives Y = z F (the DFT over n of every row m); pass 2 takes
// A = Y^T and gives Y^T F = (F Y)^T = Z^T with Z = F z F, the 2-D DFT.  The
// inverse uses Re IDFT2(G) = Re DFT2(conj G) / S^2 on the dense coefficients
// of the block (built after the loop from its pick list).
//
// Mapping.  One warp per block as in the SIMT kernels; the warps of a CTA
// form groups of four (w & ~3 .. (w & ~3) + 3), and a group's transforms run
// together: each warp stages its block's 32 rows of A in its own W area, the
// four areas form one M = 128 operand (one descriptor, 8-row groups a
// quarter of a warp area apart), the group's first warp issues the MMAs
// (N = 64, accumulators in the group's 64 tensor-memory columns), and warp
// w reads its rows back from lane quarter w & 3.  A warp that reaches a
// transform waits (bounded) for the other three to reach one too (forward
// or inverse, both are the same two GEMM passes); a warp without blocks
// left takes part in the group's transforms with rows nobody reads, until
// no warp of the group needs one.  A staging: K-major, no swizzle, core
// matrices of 8 rows x 16 B, 144 B apart along K (conflict-free column
// writes).  B (the 64 x 64 real DFT matrix, K-major) is a CTA table.
#pragma once

#include "fsr_block.cuh"

namespace fsrk {

constexpr int kWarpsTc = 12;          // 3 groups of 4 warps, one CTA per SM
constexpr int kTcMaxIters = 256;      // pick-list capacity per warp
constexpr unsigned kStatusMmaWait = 2u;   // a bounded wait on a tensor-core MMA gave up

struct TcLayout {
    // CTA tables: w0, w_f, cos/sin (as SmemLayout<float>), then the DFT matrix
    static constexpr size_t w0_off = 0;
    static constexpr size_t wf_off = w0_off + sizeof(float) * S * S;
    static constexpr size_t cs_off = wf_off + sizeof(float) * S * WFS;
    static constexpr size_t tab_off = (cs_off + sizeof(float2) * S + 127) & ~(size_t)127;
    static constexpr size_t tab_bytes = 16384;   // TF32 64 x 64 x 4 B, or BF16 hi + lo 2 x 64 x 64 x 2 B
    static constexpr size_t warp0_off = tab_off + tab_bytes;
    static constexpr size_t per_warp = SmemLayout<float>::per_warp;   // W rows + published row
    static constexpr size_t w_elems = SmemLayout<float>::w_elems;
    static constexpr size_t picks_off = warp0_off + per_warp * kWarpsTc;
    static constexpr size_t picks_per_warp = (sizeof(float2) + sizeof(int16_t)) * kTcMaxIters;
    static constexpr int groups = kWarpsTc / 4;
    static constexpr size_t bars_off = picks_off + picks_per_warp * kWarpsTc;   // tile mbarrier per warp
    static constexpr size_t gbars_off = bars_off + 8 * kWarpsTc;              // arrive + MMA mbarrier per group
    static constexpr size_t words_off = gbars_off + 16 * groups;              // tile parity per warp
    static constexpr size_t flags_off = words_off + 4 * kWarpsTc;             // "needs this pass", 2 x per warp
    static constexpr size_t tmem_off = flags_off + 8 * kWarpsTc;              // allocated TMEM base
    static constexpr size_t bytes = (tmem_off + 4 + 127) & ~(size_t)127;
    static_assert(kWarpsTc % 4 == 0, "warps form groups of four");
    static_assert(warp0_off % 128 == 0 && per_warp % 64 == 0, "warp areas: 128-byte aligned, 8-row groups at 1/4");
    static_assert(bars_off % 8 == 0, "mbarriers need 8-byte alignment");
};

// A staging within a warp area: 8-row group g at g * SBO_A, core matrices of
// 8 rows x 16 B along K at LBO_A; BF16 lo matrix at +LO_A from hi.
constexpr uint32_t SBO_A = (uint32_t)(TcLayout::per_warp / 4);
constexpr uint32_t LBO_A = 144;
constexpr uint32_t LO_A = 8 * LBO_A;   // 8 chunks of 8 BF16 per row group
// B table: 8-row groups of 64 K-elements (16 chunks of 4 TF32 or 8 of 8 BF16)
constexpr uint32_t LBO_B = 128;
template <Dft D> struct TcB;
template <> struct TcB<Dft::TF32> { static constexpr uint32_t sbo = 2048, lo = 0; };
template <> struct TcB<Dft::BF16X3> { static constexpr uint32_t sbo = 1024, lo = 8192; };
static_assert(3 * SBO_A + 16 * LBO_A <= sizeof(float2) * SmemLayout<float>::w_elems, "A staging fits the W rows");

// Instruction descriptors: D FP32, A and B K-major, N = 64, M = 128;
// A/B format TF32 (kind::tf32) or BF16 (kind::f16).
constexpr uint32_t idesc(uint32_t ab_format) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t kIdescTf32 = idesc(2);
constexpr uint32_t kIdescBf16 = idesc(1);

// Shared-memory matrix descriptor: start, leading (K) and stride (8-row)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <Dft D>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    if constexpr (D == Dft::TF32) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(d_tmem), "l"(a), "l"(b), "r"(kIdescTf32), "r"(accumulate)
                     : "memory");
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(d_tmem), "l"(a), "l"(b), "r"(kIdescBf16), "r"(accumulate)
                     : "memory");
    }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive FP32 columns of this lane's TMEM row
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ uint16_t bf16_bits(float x) {
    uint16_t r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float bf16_value(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// The CTA's B table: row nn (output column of M, 0..63), K index kk (0..63),
// value M[kk][nn] = [[cos, -sin], [sin, cos]] of t = (kk mod 32)(nn mod 32).
template <Dft D>
__device__ __forceinline__ void tc5_table(unsigned char* tab) {
    constexpr int T = (D == Dft::TF32) ? 4 : 8;   // K elements per 16-byte chunk
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int nn = i / 64, kk = i % 64;
        const int t = ((kk & 31) * (nn & 31)) & 31;
        const float c = (float)cos_2pi32(t), sn = (float)sin_2pi32(t);
        const float v = (kk < 32) ? ((nn < 32) ? c : -sn) : ((nn < 32) ? sn : c);
        const size_t off = (size_t)(nn >> 3) * TcB<D>::sbo + (size_t)(kk / T) * LBO_B + (nn & 7) * 16;
        if constexpr (D == Dft::TF32) {
            *reinterpret_cast<uint32_t*>(tab + off + (kk % T) * 4) = tf32_bits(v);
        } else {
            const uint16_t h = bf16_bits(v);
            *reinterpret_cast<uint16_t*>(tab + off + (kk % T) * 2) = h;
            *reinterpret_cast<uint16_t*>(tab + TcB<D>::lo + off + (kk % T) * 2) = bf16_bits(v - bf16_value(h));
        }
    }
}

// Bounded spin on an mbarrier phase (group syncs and MMA completions are a
// few microseconds apart, too short for a suspending wait): gives up after
// about a second of SM clock; warp-uniform result.
__device__ __forceinline__ bool spin_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    uint32_t done = 0;
    for (;;) {
        if (!done)
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(parity)
                : "memory");
        if (__all_sync(FULL, done != 0)) return true;
        if (clock64() - t0 > (2ll << 30)) return false;
    }
}

// Arrive (release) on an mbarrier without taking part in its transaction count.
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Transform context of one warp; the group's state is shared.
template <Dft D>
struct Tc5 {
    uint32_t a_grp;    // shared address of the group's 128-row A operand (W area of warp w & ~3)
    uint32_t tab;      // shared address of the B table
    uint32_t d_tmem;   // TMEM address of the group's D (lane 0, its 64 columns)
    uint32_t ld_tmem;  // TMEM address of this warp's rows (its lane quarter, the group's columns)
    uint32_t arrive;   // group mbarrier: the four warps have staged their rows (count 4)
    uint32_t mma;      // group mbarrier: the pass's MMAs have completed (count 1)
    uint32_t ph_arrive, ph_mma;   // phase parities this warp waits for next (the same in every warp of the group)
    volatile int* flags;          // the group's "needs this pass" flags, [arrive phase][4]
    unsigned* status;
    float2* zb;        // this warp's W area (A staging, transpose buffer)
    int q;             // warp index in the group
    bool ok;           // no bounded wait has given up

    // lane n holds column n of the 32 x 32 complex input in (cr, ci): stage
    // A[m][n] = cr[m], A[m][32 + n] = ci[m] (rows m of this warp)
    __device__ __forceinline__ void stage(const float (&cr)[S], const float (&ci)[S], int lane) {
        unsigned char* base = reinterpret_cast<unsigned char*>(zb);
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const size_t row = (size_t)(m >> 3) * SBO_A + (m & 7) * 16;
            if constexpr (D == Dft::TF32) {
                const int k0 = lane, k1 = 32 + lane;
                *reinterpret_cast<uint32_t*>(base + row + (k0 >> 2) * LBO_A + (k0 & 3) * 4) = tf32_bits(cr[m]);
                *reinterpret_cast<uint32_t*>(base + row + (k1 >> 2) * LBO_A + (k1 & 3) * 4) = tf32_bits(ci[m]);
            } else {
                const int k0 = lane, k1 = 32 + lane;
                const uint16_t hr = bf16_bits(cr[m]), hi = bf16_bits(ci[m]);
                const size_t o0 = row + (k0 >> 3) * LBO_A + (k0 & 7) * 2, o1 = row + (k1 >> 3) * LBO_A + (k1 & 7) * 2;
                *reinterpret_cast<uint16_t*>(base + o0) = hr;
                *reinterpret_cast<uint16_t*>(base + o1) = hi;
                *reinterpret_cast<uint16_t*>(base + LO_A + o0) = bf16_bits(cr[m] - bf16_value(hr));
                *reinterpret_cast<uint16_t*>(base + LO_A + o1) = bf16_bits(ci[m] - bf16_value(hi));
            }
        }
    }

    // One GEMM pass of the group: D (128 x 64) = A . M.  ACTIVE: this warp
    // staged rows it needs; it then receives row r of its block's D in
    // (vr, vi) = columns 0..31, 32..63.  Returns the number of warps of the
    // group that needed the pass (0: no MMA was issued, possible only for an
    // idle warp); -1 when a bounded wait gave up (the warp marks itself
    // failed).
    template <bool ACTIVE>
    __device__ __forceinline__ int pass(float (&vr)[32], float (&vi)[32], int lane) {
        if (!ok) return -1;
        // rows staged by this warp (generic proxy) become visible to the MMA
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        // flags of consecutive passes alternate between two sets: a warp can
        // be at most one pass ahead of the slowest reader
        volatile int* f = flags + 4 * ph_arrive;
        if (lane == 0) {
            f[q] = ACTIVE ? 1 : 0;
            bar_arrive(arrive);
        }
        if (!spin_wait(arrive, ph_arrive)) {
            if (lane == 0) atomicOr(status, kStatusMmaWait);
            ok = false;
            return -1;
        }
        ph_arrive ^= 1u;
        const int n = f[0] + f[1] + f[2] + f[3];
        if constexpr (!ACTIVE) {
            if (n == 0) return 0;
        }
        if (q == 0 && lane == 0) {
            tc_fence_after();
            if constexpr (D == Dft::TF32) {
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    tc_mma<D>(d_tmem, smem_desc(a_grp + ks * 2 * LBO_A, LBO_A, SBO_A),
                              smem_desc(tab + ks * 2 * LBO_B, LBO_B, TcB<D>::sbo), ks > 0);
            } else {
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ah = a_grp + ks * 2 * LBO_A, bh = tab + ks * 2 * LBO_B;
                    tc_mma<D>(d_tmem, smem_desc(ah + LO_A, LBO_A, SBO_A), smem_desc(bh, LBO_B, TcB<D>::sbo), ks > 0);
                    tc_mma<D>(d_tmem, smem_desc(ah, LBO_A, SBO_A), smem_desc(bh + TcB<D>::lo, LBO_B, TcB<D>::sbo), 1);
                    tc_mma<D>(d_tmem, smem_desc(ah, LBO_A, SBO_A), smem_desc(bh, LBO_B, TcB<D>::sbo), 1);
                }
            }
            tc_commit(mma);
        }
        __syncwarp();
        if (!spin_wait(mma, ph_mma)) {
            if (lane == 0) atomicOr(status, kStatusMmaWait);
            ok = false;
            return -1;
        }
        ph_mma ^= 1u;
        tc_fence_after();
        if constexpr (ACTIVE) {
            tc_ld32(ld_tmem, vr);
            tc_ld32(ld_tmem + 32u, vi);
        }
        return n;
    }

    // 2-D DFT: lane n holds column n of the input in (zr, zi); on return lane
    // k holds row k of Z = DFT2(input) in (zr, zi).  False when a wait gave
    // up (the result is then not valid).
    __device__ __forceinline__ bool dft2(float (&zr)[S], float (&zi)[S], int lane) {
        float yr[S], yi[S];
        __syncwarp();
        stage(zr, zi, lane);
        if (pass<true>(yr, yi, lane) < 0) return false;   // lane m: Y[m][0..31]
        __syncwarp();
        stage(yr, yi, lane);                               // A2 = Y^T: lane m writes column m
        if (pass<true>(zr, zi, lane) < 0) return false;   // lane l: Z[0..31][l]
        // transpose through the W area: lane k receives row k of Z
        __syncwarp();
#pragma unroll
        for (int k = 0; k < S; ++k) zb[k * TSTRIDE + lane] = make_float2(zr[k], zi[k]);
        __syncwarp();
#pragma unroll
        for (int l = 0; l < S; ++l) {
            const float2 t = zb[lane * TSTRIDE + l];
            zr[l] = t.x;
            zi[l] = t.y;
        }
        __syncwarp();
        return true;
    }

    // A warp without blocks left: take part in the group's passes (two per
    // transform) until no warp of the group needs one.
    __device__ __forceinline__ void idle(int lane) {
        float vr[32], vi[32];
        for (;;) {
            if (pass<false>(vr, vi, lane) <= 0) return;
            if (pass<false>(vr, vi, lane) < 0) return;
        }
    }
};

// a9 on tensor cores: the dense coefficients Gc (G of Eq. 11 over S^2) from
// the block's pick list (every entry summed in iteration order), then
// Re g = Re DFT2(conj Gc); the B x B target values are gathered into gacc
// (target pixel t is (L + t / B, L + t % B), L = (S - B) / 2).
template <int B, Dft D>
__device__ __forceinline__ void tc5_inverse_targets(Tc5<D>& tc, const PickList& pl, int K, float2* rowbuf, int lane,
                                                    float (&zr)[S], float (&zi)[S], float (&gacc)[TargetPix<B>::P]) {
    constexpr int LB = (S - B) / 2;
    float2* gc = tc.zb;   // 32 x 32 dense coefficients in the (now free) W area
    __syncwarp();
#pragma unroll
    for (int l = 0; l < S; ++l) gc[lane * S + l] = make_float2(0.f, 0.f);
    __syncwarp();
    for (int nu = 0; nu < K; ++nu) {   // lane u sums the picks of its row in order
        const int idx = pl.idx[nu];
        if ((idx >> 5) == lane) {
            const float2 c = pl.c[nu];
            float2 g = gc[idx];
            g.x += c.x;
            g.y += c.y;
            gc[idx] = g;
        }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < S; ++m) {   // lane n: column n of conj(Gc)
        const float2 g = gc[m * S + lane];
        zr[m] = g.x;
        zi[m] = -g.y;
    }
    if (!tc.dft2(zr, zi, lane)) return;   // lane k: row k
    float* tb = reinterpret_cast<float*>(rowbuf);
    if (lane >= LB && lane < LB + B) {
#pragma unroll
        for (int c = 0; c < B; ++c) tb[(lane - LB) * B + c] = zr[LB + c];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < TargetPix<B>::P; ++q) {
        const int pidx = lane + 32 * q;
        gacc[q] = pidx < B * B ? tb[pidx] : 0.f;
    }
    __syncwarp();
}

// Single image, B = 4, one CTA of kWarpsTc warps per SM, dynamic block
// counter; K <= kTcMaxIters.
template <Dft D>
__global__ void __launch_bounds__(kWarpsTc * 32, 1) fsr_tc_kernel(const __grid_constant__ KernelArgs a) {
    constexpr int B = 4;
    constexpr int P = TargetPix<B>::P;
    using Lay = TcLayout;
    extern __shared__ __align__(128) unsigned char smem[];
    float* sw0 = reinterpret_cast<float*>(smem + Lay::w0_off);
    float* swf = reinterpret_cast<float*>(smem + Lay::wf_off);
    float2* scs = reinterpret_cast<float2*>(smem + Lay::cs_off);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float2* Wd = reinterpret_cast<float2*>(smem + Lay::warp0_off + Lay::per_warp * warp);
    float2* rowbuf = Wd + Lay::w_elems;
    uint32_t* words = reinterpret_cast<uint32_t*>(smem + Lay::words_off);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Lay::tmem_off);
    const int grp = warp >> 2;

    cta_tables<float>(a.mth, sw0, swf, scs);
    tc5_table<D>(smem + Lay::tab_off);
    const uint32_t tile_bar = smem_addr(smem + Lay::bars_off + 8 * warp);
    const uint32_t arrive_bar = smem_addr(smem + Lay::gbars_off + 16 * grp);
    const uint32_t mma_bar = arrive_bar + 8;
    if (lane == 0) {
        tile_bar_init(tile_bar);
        words[warp] = 0;   // tile phase parity
        if ((warp & 3) == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(arrive_bar) : "memory");
            tile_bar_init(mma_bar);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if (warp == 0) {   // 64 columns per group of four warps
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    Tc5<D> tc;
    tc.a_grp = smem_addr(smem + Lay::warp0_off + Lay::per_warp * (warp & ~3));
    tc.tab = smem_addr(smem + Lay::tab_off);
    tc.d_tmem = tmem + 64u * grp;
    tc.ld_tmem = tmem + ((32u * (warp & 3)) << 16) + 64u * grp;
    tc.arrive = arrive_bar;
    tc.mma = mma_bar;
    tc.ph_arrive = 0;
    tc.ph_mma = 0;
    tc.flags = reinterpret_cast<volatile int*>(smem + Lay::flags_off) + 8 * grp;
    tc.status = a.status;
    tc.zb = Wd;
    tc.q = warp & 3;
    tc.ok = true;
    PickList pl;
    pl.c = reinterpret_cast<float2*>(smem + Lay::picks_off + Lay::picks_per_warp * warp);
    pl.idx = reinterpret_cast<int16_t*>(pl.c + kTcMaxIters);

    const bool tiles = a.tiles && (smem_addr(smem) & 127u) == 0;
    const float gamma = a.mth.gamma;
    const int L = a.mth.L;
    for (;;) {
        unsigned long long next = 0;
        if (lane == 0) next = atomicAdd(a.work, 1ull);
        const long long blk = (long long)__shfl_sync(FULL, next, 0);
        if (blk >= a.nblocks || !tc.ok) break;
        const ImageArgs& im = a.im;
        const int by = (int)(blk / im.nbx);
        const int bx = (int)(blk - (long long)by * im.nbx);
        const int y0 = by * B - L, x0 = bx * B - L;
        const unsigned char* tile = nullptr;
        if (tiles) {
            __syncwarp();
            if (lane == 0) tile_issue(&a.maps, smem_addr(Wd), tile_bar, y0, x0, kTileBytes + (unsigned)a.tx_extra);
            const uint32_t parity = words[warp];
            if (!tile_wait(tile_bar, parity)) {
                if (lane == 0) atomicOr(a.status, kStatusTileWait);
                break;
            }
            __syncwarp();
            if (lane == 0) words[warp] = parity ^ 1u;
            tile = reinterpret_cast<const unsigned char*>(Wd);
        }
        float zr[S], zi[S];
        BlockState<float> st;
        float gacc[P];
#pragma unroll
        for (int q = 0; q < P; ++q) gacc[q] = 0.f;
        int16_t* seq = im.seq ? im.seq + (size_t)blk * im.K : nullptr;
        if (prepare_block<float, SmemLayout<float>::WS, D, false, Tc5<D>>(im, y0, x0, lane, sw0, Wd, &tc, tile, zr,
                                                                          zi, st)) {
            iterate<B, true>(zr, zi, Wd, rowbuf, swf, scs, st, gamma, im.K, L, lane, seq, gacc, &pl);
            tc5_inverse_targets<B, D>(tc, pl, im.K, rowbuf, lane, zr, zi, gacc);
        } else if (lane == 0) {
            empty_block(seq, im.K, a.empty);
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int pidx = lane + 32 * q;
            if (pidx < B * B) {
                const int ty = by * B + pidx / B, tx = bx * B + pidx % B;
                if (ty < im.H && tx < im.W) {
                    const size_t off = (size_t)ty * im.pitch + tx;
                    const bool kn = __ldg(im.mask + off) != 0;
                    im.out[off] = kn ? __ldg(im.img + off) : gacc[q];
                }
            }
        }
    }
    // no blocks left: take part in the group's transforms until none needs one
    tc.idle(lane);
    // after a wait that gave up, wait once more (bounded) for MMAs in flight
    // before the tensor memory is released
    if (!tc.ok) spin_wait(tc.mma, tc.ph_mma);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
    // the last warp of the launch leaves the counter at zero for the next one
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(a.work + 1, 1ull) == (unsigned long long)gridDim.x * kWarpsTc - 1) {
            atomicExch(a.work, 0ull);
            atomicExch(a.work + 1, 0ull);
        }
    }
}

}  // namespace fsrk
