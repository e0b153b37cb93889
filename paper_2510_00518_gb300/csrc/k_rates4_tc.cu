// k_rates4_tc.cu - four-phonon +- channel, mixed precision, two-atom cells, with the cluster
// contraction X = Σ_r P_r^s2 W_r on the tensor cores (tcgen05).
//
// Persistent CTAs of 384 threads (one per SM: they hold all 512 TMEM columns) loop over units
// (λ, q').  On the triangular domain a unit first lists its q'' <= q''' (block scan, ascending);
// the rounds then run over that list.  For a round of 128 partner points q'' the contraction of
// every (c, d) key group is one real matrix product covering all partner branches j':
//   [Xr | Xi](q'', j' γδ) = [Pr | s2 Pi](q'', r) . [[Wr, Wi], [-Wi, Wr]](r, j' γδ)
// (rows q'' = MMA M = 128 = TMEM lanes; K = 2 x keys of the group, padded to 16; N = 112 columns
// of which 108 hold the 6 x 9 complex (j', γδ)).  The FP32 operands enter the tensor cores in one
// of four formats (W scaled by a power of two per unit so that max |W| < 1):
//   FP16 x3   kind::f16, FP16 hi/lo splits, products hi.hi + hi.lo + lo.hi: ~2^-21 relative
//   BF16 x3   kind::f16 with BF16 operands, hi/lo splits, three products: ~2^-16
//   BF16      kind::f16 with BF16 operands, one product: ~2^-8 (single pass)
//   TF32 x3   kind::tf32, TF32 hi/lo splits (round to nearest), three products: ~2^-21
// all accumulating in FP32 in tensor memory.  B is built once per unit, A once per round; one
// thread issues tcgen05.mma and tcgen05.commit to an mbarrier.  The three warpgroups then share the 128 rows:
// warpgroup g reads X of partner branches j' = g and g + 3 for its row with tcgen05.ld and
// evaluates that (q'', j') entry directly (Y = X e*''' per j''', V = e''.Y per kept j'', weights:
// 2 for a swapped pair, 1 on the diagonal q'' = q''' with j'' = j''').
//
// Waits on the mbarrier are bounded (fc4_options.timeout_cycles SM clocks, default 2e9); on expiry
// the kernel sets the context's error flag (the reduction then writes NaN into Γ), waits once
// more (~1 s at most) for its MMAs in flight, writes empty partials for its remaining units, frees
// its tensor memory and returns.
#include "k_rates4.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace fc4 {

namespace {

constexpr int kTcRows = 128;                // q'' per round = MMA M = TMEM lanes
constexpr int kTcThreads = 384;             // three warpgroups over the same 128 rows
constexpr int kTcTriChunk = 4 * kTcThreads; // q'' per chunk of the triangle list
constexpr int kTcN = 112;                   // MMA N per (c, d) group: 6 j' x 18 columns used
constexpr int kTcCols = 512;                // TMEM columns: 4 groups x 112, allocated as 512

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: canonical K-major layout without swizzle (8-row x 16-byte core
// matrices stored contiguously); lbo = byte step between core matrices along K, sbo = along M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

// Operand formats of the contraction (fc4_precision of the context).
enum TcOp { kOpF16x3 = 0, kOpBF16x3 = 1, kOpBF16 = 2, kOpTF32x3 = 3 };

template <int OP>
struct TcFmt {
    static constexpr int ES = OP == kOpTF32x3 ? 4 : 2;       // bytes per element
    static constexpr int EPC = 16 / ES;                      // elements per 16-byte core-matrix row
    static constexpr int KI = 32 / ES;                       // K of one MMA instruction
    static constexpr int NPROD = OP == kOpBF16 ? 1 : 3;      // hi.hi (+ hi.lo + lo.hi)
    static constexpr int NT = NPROD > 1 ? 2 : 1;             // operand tiles: hi (and lo)
    // instruction descriptor: D FP32 (bit 4), A and B format (bits 7-9, 10-12: 0 FP16, 1 BF16,
    // 2 TF32), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t FMT = OP == kOpF16x3 ? 0u : OP == kOpTF32x3 ? 2u : 1u;
    static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) |
                                      ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
};

template <int OP>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
    if constexpr (OP == kOpTF32x3)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem), "l"(ad), "l"(bd), "r"(TcFmt<OP>::IDESC), "r"(acc) : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem), "l"(ad), "l"(bd), "r"(TcFmt<OP>::IDESC), "r"(acc) : "memory");
}

// FP32 x -> operand bits hi (and lo = the rounding of x - hi), each in the low ES bytes
template <int OP>
__device__ __forceinline__ void split_op(float x, uint32_t &hi, uint32_t &lo) {
    if constexpr (OP == kOpF16x3) {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    } else if constexpr (OP == kOpTF32x3) {
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - __uint_as_float(h)));
        hi = h;
        lo = l;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = OP == kOpBF16 ? 0u : (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    }
}

template <int ES>
__device__ __forceinline__ void store_op(unsigned char *p, uint32_t v) {
    if constexpr (ES == 4) *reinterpret_cast<uint32_t *>(p) = v;
    else *reinterpret_cast<unsigned short *>(p) = (unsigned short)v;
}

// bounded wait for the completion of phase `phase` of an mbarrier, at most max_cycles SM clocks.
// Long bounds use try_wait, which suspends the thread until the phase completes (or a ~20 us
// hint runs out); bounds below 1e5 clocks poll with test_wait so that they are honoured exactly.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long max_cycles) {
    const long long t0 = clock64();
    const bool poll = max_cycles < 100000;
    for (;;) {
        uint32_t ok;
        if (poll)
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(mbar), "r"(phase) : "memory");
        else
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(mbar), "r"(phase), "r"(20000u) : "memory");
        if (ok) return true;
        if (clock64() - t0 > max_cycles) return false;
    }
}

// 16 + 2 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld18(uint32_t addr, float (&v)[18]) {
    uint32_t r[18];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                 : "=r"(r[16]), "=r"(r[17]) : "r"(addr + 16));
#pragma unroll
    for (int k = 0; k < 18; ++k) v[k] = __uint_as_float(r[k]);
}

// byte offset of element (row, k) in a K-major no-swizzle tile with `rows` rows of ES-byte elements
template <int ES>
__device__ __forceinline__ uint32_t tile_off(int row, int k, int rows) {
    constexpr int EPC = 16 / ES;
    return 128u * (uint32_t)((k / EPC) * (rows >> 3) + (row >> 3)) + 16u * (uint32_t)(row & 7) +
           (uint32_t)ES * (uint32_t)(k % EPC);
}

}  // namespace

// Key layout of the contraction: group g = c NA + d holds keys [grp_start[g], grp_start[g+1]);
// its K extent is 2 x keys padded to the K of one MMA instruction (ki elements), at offset
// koff[g] (elements) of the K axis.
struct TcPlan {
    int kt;                   // total K (elements)
    int koff[4], kpad[4], nkey[4], r0[4];
};

__host__ __device__ inline TcPlan tc_plan(const Tables &t, int ki) {
    TcPlan p{};
    int o = 0;
    for (int g = 0; g < 4; ++g) {
        p.r0[g] = t.grp_start[g];
        p.nkey[g] = t.grp_start[g + 1] - t.grp_start[g];
        p.kpad[g] = (2 * p.nkey[g] + ki - 1) / ki * ki;
        p.koff[g] = o;
        o += p.kpad[g];
    }
    p.kt = o;
    return p;
}

// shared memory: A hi [| A lo] (128 x kt elements each) | B hi [| B lo] (112 x kt elements each)
template <int OP>
inline size_t tc_smem_bytes(const Tables &t) {
    using F = TcFmt<OP>;
    const TcPlan p = tc_plan(t, F::KI);
    return (size_t)F::NT * kTcRows * p.kt * F::ES + (size_t)F::NT * kTcN * p.kt * F::ES + 128;
}

template <bool ADA, int OP>
__global__ void __launch_bounds__(kTcThreads, 1)
rates4_tc_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch, int mode0,
                 int n_units, const float2 *__restrict__ wall) {
    constexpr int NA = 2, NB = 6, NG = 4;
    using F = TcFmt<OP>;
    constexpr int ES = F::ES;
    const int s1 = (ch == 4) ? -1 : 1;
    const int s2 = (ch == 2) ? 1 : -1;
    const int N = t.N, nk = t.n_keys;
    const TcPlan pl = tc_plan(t, F::KI);
    const uint32_t a_tile = (uint32_t)(kTcRows * ES) * pl.kt, b_tile = (uint32_t)(kTcN * ES) * pl.kt;

    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *sA = tc_smem;                                         // hi, then lo at + a_tile
    unsigned char *sB = sA + (size_t)F::NT * a_tile;                     // hi, then lo at + b_tile
    const uint32_t a_hi = smem_u32(sA), a_lo = a_hi + a_tile;
    const uint32_t b_hi = smem_u32(sB), b_lo = b_hi + b_tile;
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ double s_red[2 * 32];
    __shared__ long long s_redn[5 * 32];
    __shared__ float s_wmax[kTcThreads / 32];
    __shared__ int s_scan[32];
    __shared__ unsigned short s_tri[kTcTriChunk];               // triangle: q'' - chunk start

    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kTcRows - 1), wg = tid >> 7;         // TMEM lane = row; warpgroup
    constexpr int nj = 2;                                       // partner branches per warpgroup: g, g + 3
    const float2 *ev = t.ev32;
    const float *occ = t.occ32;
    const float *invw = t.invw32;
    const long long spins = a.spin_limit > 0 ? a.spin_limit : 2000000000ll;   // ~1 s
    const uint32_t mbar = smem_u32(&s_mbar);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // B padding (rows 108..111, K columns beyond 2 x keys) stays zero for the whole kernel
    for (int k = tid; k < (int)(F::NT * b_tile / 4); k += kTcThreads) reinterpret_cast<uint32_t *>(sB)[k] = 0u;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    uint32_t phase = 0;
    bool dead = false;
    int unit = blockIdx.x;

    for (; unit < n_units && !dead; unit += gridDim.x) {
        const int ml = unit / N, q1 = unit - ml * N;
        const int ms = mode0 + ml;
        const int m0 = a.modes[ms];
        const int q0 = m0 / NB, j0 = m0 - q0 * NB;
        Acc<float> acc_g, acc_wp;
        long long acc_n = 0, acc_items = 0, acc_ent = 0, acc_ev = 0, acc_cev = 0;
        const unsigned vm1 = t.vmask[q1];
        if (!(q0 == 0 && j0 < 3) && vm1) {                       // uniform across the block
            const float2 *wsrc = wall + (size_t)unit * (NB * nk * 9);
            float mx = 0.0f;
            for (int k = tid; k < NB * nk * 9; k += kTcThreads) {
                const float2 w = wsrc[k];
                mx = fmaxf(mx, fmaxf(fabsf(w.x), fabsf(w.y)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            if ((tid & 31) == 0) s_wmax[warp] = mx;
            __syncthreads();                                     // also: the previous unit is done
            int e_w = 0;
            {
                float m = 0.0f;
                for (int w = 0; w < kTcThreads / 32; ++w) m = fmaxf(m, s_wmax[w]);
                if (m > 0.0f) frexpf(m, &e_w);
            }
            const float wscale = ldexpf(1.0f, -e_w), xscale = ldexpf(1.0f, e_w);
            // B of the unit: row n = 18 j' + 2 γδ + (0 re, 1 im) of every group, FP16 hi / lo
            for (int k = tid; k < NB * nk * 9; k += kTcThreads) {
                const int j1 = k / (nk * 9), rem = k - j1 * (nk * 9);
                const int r = rem / 9, gd = rem - r * 9;
                int g = 0;
#pragma unroll
                for (int gg = 1; gg < NG; ++gg) g += (r >= pl.r0[gg]);
                const int kr = r - pl.r0[g];
                const float2 w = wsrc[k];
                const float wr = w.x * wscale, wi = w.y * wscale;
                const float val[4] = {wr, -wi, wi, wr};        // (re row: k, K + k), (im row: k, K + k)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int n = 18 * j1 + 2 * gd + (u >> 1);
                    const int kk = pl.koff[g] + kr + ((u & 1) ? pl.nkey[g] : 0);
                    uint32_t h, l;
                    split_op<OP>(val[u], h, l);
                    const uint32_t off = tile_off<ES>(n, kk, kTcN);
                    store_op<ES>(sB + off, h);
                    if constexpr (F::NT > 1) store_op<ES>(sB + b_tile + off, l);
                }
            }

            const int4 c0 = t.qc[q0], c1 = t.qc[q1];
            const int b0 = c0.x + s1 * c1.x, b1 = c0.y + s1 * c1.y, b2 = c0.z + s1 * c1.z;
            const double w0 = t.om[m0];
            const float w0f = t.om32[m0];

            // On the triangle the rounds take only the q'' <= q''' (a list per chunk of q'', in
            // ascending order), so the MMA, the A staging and the TMEM reads of the skipped half go too.
            const bool pm_list = (a.tri & 1) != 0;
            for (int cb = 0; cb < N && !dead; cb += pm_list ? kTcTriChunk : N) {
              int cnt = N - cb;
              if (pm_list) {
                constexpr int kPer = kTcTriChunk / kTcThreads;
                const int ce = min(N, cb + kTcTriChunk), lo = cb + tid * kPer;
                unsigned fl = 0;
                int nf = 0;
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int qq = lo + i;
                    if (qq < ce) {
                        const int4 c2 = t.qc[qq];
                        const int qr = q_index_near(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z,
                                                    t.mesh[0], t.mesh[1], t.mesh[2]);
                        if (qq <= qr) { fl |= 1u << i; ++nf; }
                    }
                }
                int off = block_exclusive_scan(nf, s_scan, &cnt);
#pragma unroll
                for (int i = 0; i < kPer; ++i)
                    if ((fl >> i) & 1u) s_tri[off++] = (unsigned short)(tid * kPer + i);
                __syncthreads();
              }
              for (int qb = 0; qb < cnt && !dead; qb += kTcRows) {
                const int ix = qb + row;
                const bool valid = ix < cnt;
                const int q2 = valid ? cb + (pm_list ? (int)s_tri[ix] : ix) : 0;
                // A: row `row`, the warpgroup's groups (0 | 1, 2 | 3: its share of the row), FP16 hi / lo
                const float2 *Prow = t.P4_32 + (size_t)(valid ? q2 : 0) * nk;
                for (int g = (wg == 0 ? 0 : wg == 1 ? 1 : 3); g <= (wg == 0 ? 0 : wg == 1 ? 2 : 3); ++g) {
                    // one 16-byte core-matrix row (F::EPC consecutive K elements) per store: the 32
                    // rows of a warp write 512 contiguous bytes, free of bank conflicts
                    for (int k = 0; k < pl.kpad[g]; k += F::EPC) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int w = 0; w < 4; ++w) { hw[w] = 0u; lw[w] = 0u; }
#pragma unroll
                        for (int u = 0; u < F::EPC; ++u) {
                            const int kk = k + u;
                            float x = 0.0f;
                            if (valid && kk < 2 * pl.nkey[g]) {
                                const float2 p = Prow[pl.r0[g] + (kk < pl.nkey[g] ? kk : kk - pl.nkey[g])];
                                x = kk < pl.nkey[g] ? p.x : (float)s2 * p.y;
                            }
                            uint32_t h, l;
                            split_op<OP>(x, h, l);
                            const int sh = (u * ES * 8) & 31, wi = (u * ES) >> 2;
                            hw[wi] |= h << sh;
                            lw[wi] |= l << sh;
                        }
                        const uint32_t off = tile_off<ES>(row, pl.koff[g] + k, kTcRows);
                        *reinterpret_cast<uint4 *>(sA + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if constexpr (F::NT > 1)
                            *reinterpret_cast<uint4 *>(sA + a_tile + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                // window of this row for the warpgroup's partner branches: bit NB j3 + j2 set iff kept
                unsigned long long keep[2] = {0ull, 0ull};
                int q3 = 0, tri = -1;
                if (valid) {
                    const int4 c2 = t.qc[q2];
                    q3 = q_index_near(b0 + s2 * c2.x, b1 + s2 * c2.y, b2 + s2 * c2.z, t.mesh[0], t.mesh[1], t.mesh[2]);
                    const unsigned v2 = t.vmask[q2], v3 = t.vmask[q3];
                    float w2f[NB], w3f[NB];
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        w2f[j] = (float)s2 * t.om32[q2 * NB + j];
                        w3f[j] = t.om32[q3 * NB + j];
                    }
                    // triangular domain of +- (λ'' <-> λ'''), as in the CUDA-core kernels
                    tri = tri_code_sampled(a, ch, m0, q1, q2, q3, N);
                    unsigned long long okm = 0;
#pragma unroll
                    for (int j3 = 0; j3 < NB; ++j3)
                        if ((v3 >> j3) & 1u) {
                            unsigned row = v2 & ((1u << NB) - 1u);
                            if (tri == 2) row &= (2u << j3) - 1u;        // j'' <= j'''
                            okm |= (unsigned long long)row << (NB * j3);
                        }
                    if (tri < 0) okm = 0;                                // the swap of another row
                    else acc_cev += (long long)nj * NB * NB;
                    if constexpr (ADA) {
                        // the width of a pair (λ'', λ''') is formed once for both partner branches
#pragma unroll 1
                        for (int j3 = 0; j3 < NB; ++j3) {
                            if (!((v3 >> j3) & 1u)) continue;
                            const int m3 = q3 * NB + j3;
                            const float4 h3 = t.vp32[m3], l3 = t.vp32lo[m3];
                            float g32[NB];
#pragma unroll
                            for (int j2 = 0; j2 < NB; ++j2)
                                g32[j2] = a.ad_c32 * vel_diff_norm32(t.vp32[q2 * NB + j2], t.vp32lo[q2 * NB + j2], h3, l3);
#pragma unroll
                            for (int jj = 0; jj < nj; ++jj) {
                                const int j1 = wg + 3 * jj;
                                if (!((vm1 >> j1) & 1u)) continue;
                                const float b = w0f + (float)s1 * t.om32[q1 * NB + j1];
                                unsigned row = 0;
#pragma unroll
                                for (int j2 = 0; j2 < NB; ++j2) {
                                    if (!((v2 >> j2) & 1u)) continue;
                                    const float ad = fabsf((b + w2f[j2]) - w3f[j3]);
                                    const int w = window_adaptive32(a, ad, g32[j2]);
                                    if (w == 2 || (w == 1 && window_exact_adaptive(t, a, ch, m0, q1 * NB + j1, q2 * NB + j2,
                                                                                     m3, q2 * NB + j2, m3)))
                                        row |= 1u << j2;
                                }
                                keep[jj] |= (unsigned long long)row << (NB * j3);
                            }
                        }
#pragma unroll
                        for (int jj = 0; jj < nj; ++jj) keep[jj] &= okm;
                    }
#pragma unroll
                    for (int jj = 0; jj < nj; ++jj) {
                        const int j1 = wg + 3 * jj;
                        if (!((vm1 >> j1) & 1u)) continue;
                        const float b = w0f + (float)s1 * t.om32[q1 * NB + j1];
                        if constexpr (ADA) {
                        } else {
                            float t2[NB];
#pragma unroll
                            for (int j2 = 0; j2 < NB; ++j2) t2[j2] = b + w2f[j2];
                            unsigned long long le_lo = 0, le_hi = 0;
#pragma unroll
                            for (int j3 = 0; j3 < NB; ++j3)
#pragma unroll
                                for (int j2 = 0; j2 < NB; ++j2) {
                                    const float ad = fabsf(t2[j2] - w3f[j3]);
                                    le_lo |= (unsigned long long)(ad <= a.lo32) << (NB * j3 + j2);
                                    le_hi |= (unsigned long long)(ad <= a.hi32) << (NB * j3 + j2);
                                }
                            unsigned long long sure = le_lo & okm, amb = le_hi & ~le_lo & okm;
                            while (amb) {
                                const int k = __ffsll(amb) - 1;
                                amb &= amb - 1;
                                const int j3 = k / NB, j2 = k - j3 * NB;
                                if (window_exact4(ch, w0, t.om[q1 * NB + j1], t.om[q2 * NB + j2],
                                                  t.om[q3 * NB + j3], a.two_sigma))
                                    sure |= 1ull << k;
                            }
                            keep[jj] = sure;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                const int any = __syncthreads_or((keep[0] | keep[1]) != 0ull);
                if (!any) continue;                              // no entry in this round
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        for (int pz = 0; pz < F::NPROD; ++pz) {  // hi.hi (, hi.lo, lo.hi)
                            const uint32_t ab = (pz == 2 ? a_lo : a_hi) + (uint32_t)(kTcRows * ES) * pl.koff[g];
                            const uint32_t bb = (pz == 1 ? b_lo : b_hi) + (uint32_t)(kTcN * ES) * pl.koff[g];
                            for (int s = 0; s < pl.kpad[g] / F::KI; ++s)
                                mma_issue<OP>(tmem + (uint32_t)(kTcN * g), smem_desc(ab + 4096u * s, 2048u, 128u),
                                              smem_desc(bb + 3584u * s, 1792u, 128u), (pz > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(mbar) : "memory");
                }
                const bool ok = mbar_wait(mbar, phase, spins);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {                     // the MMAs did not complete
                    if (tid == 0 && a.err) atomicExch(a.err, 1);
                    mbar_wait(mbar, phase ^ 1u, 2000000000ll);   // let the MMAs in flight finish
                    dead = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int iq2 = q2, iq3 = q3;
                for (int jj = 0; jj < nj; ++jj) {
                    const int j1 = wg + 3 * jj;
                    // this row's X for partner branch j1 (warp-collective loads)
                    float xr[NG][18];
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (pl.nkey[g] == 0) {
#pragma unroll
                            for (int k = 0; k < 18; ++k) xr[g][k] = 0.0f;
                        } else {
                            tmem_ld18(tmem + lane_base + (uint32_t)(kTcN * g + 18 * j1), xr[g]);
                        }
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    const unsigned long long e = keep[jj];
                    if (!e) continue;
                    ++acc_ent;
                    const int m1 = q1 * NB + j1;
                    float ee1;
                    const float ex1 = two_sum(t.om32[m0], (float)s1 * t.om32[m1], ee1);
                    const float el01 = t.om32lo[m0] + (float)s1 * t.om32lo[m1];
                    const float iw01 = invw[m0] * invw[m1];
                    const float n1f = occ[m1];
                    float2 X[NA][NA][9];
#pragma unroll
                    for (int c = 0; c < NA; ++c)
#pragma unroll
                        for (int d = 0; d < NA; ++d)
#pragma unroll
                            for (int k = 0; k < 9; ++k)
                                X[c][d][k] = make_float2(xr[c * NA + d][2 * k] * xscale, xr[c * NA + d][2 * k + 1] * xscale);
#pragma unroll 1
                    for (int j3 = 0; j3 < NB; ++j3) {
                        unsigned m = (unsigned)(e >> (NB * j3)) & ((1u << NB) - 1u);
                        if (!m) continue;
                        ++acc_items;
                        float2 Y[NA][3];
#pragma unroll
                        for (int c = 0; c < NA; ++c)
#pragma unroll
                            for (int g = 0; g < 3; ++g) Y[c][g] = czero<float2>();
#pragma unroll
                        for (int d = 0; d < NA; ++d) {
                            float2 e3[3];
#pragma unroll
                            for (int dl = 0; dl < 3; ++dl) e3[dl] = cconj(ev[(iq3 * NB + 3 * d + dl) * NB + j3]);
#pragma unroll
                            for (int c = 0; c < NA; ++c)
#pragma unroll
                                for (int g = 0; g < 3; ++g)
#pragma unroll
                                    for (int dl = 0; dl < 3; ++dl) Y[c][g] = cfma(X[c][d][3 * g + dl], e3[dl], Y[c][g]);
                        }
                        const int m3 = iq3 * NB + j3;
                        const float n3 = occ[m3], iw3 = invw[m3];
                        const float h3 = t.om32[m3], l3 = t.om32lo[m3];
                        while (m) {
                            const int j2 = __ffs(m) - 1;
                            m &= m - 1;
                            const int m2 = iq2 * NB + j2;
                            float2 V = czero<float2>();
#pragma unroll
                            for (int c = 0; c < NA; ++c)
#pragma unroll
                                for (int g = 0; g < 3; ++g)
                                    V = cfma(cconj_if(ev[(iq2 * NB + 3 * c + g) * NB + j2], s2 < 0), Y[c][g], V);
                            float e2s, e3s;
                            const float x2 = two_sum(ex1, (float)s2 * t.om32[m2], e2s);
                            const float x3 = two_sum(x2, -h3, e3s);
                            const float lo = (el01 + (float)s2 * t.om32lo[m2]) - l3;
                            const float df = x3 + ((ee1 + e2s) + (e3s + lo));
                            float gs;
                            if constexpr (ADA) gs = gauss_adaptive32(t, a, df, m2, m3);
                            else gs = __expf(-(df * df) * a.inv_sigma2_32) * a.gnorm32;
                            const float w = sym4<float>(ch) * occupation_factor<float>(ch, n1f, occ[m2], n3) * gs *
                                            iw01 * (invw[m2] * iw3);
                            const int wt = tri_weight(tri, j1, j2, j3);
                            acc_wp.add(w * (float)wt);
                            acc_g.add((w * (float)wt) * (V.x * V.x + V.y * V.y));
                            acc_n += wt;
                            acc_ev += 1;
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();                                 // A and TMEM are reused next round
              }
            }
        }
        double sums[2] = {acc_g.value(), acc_wp.value()};
        long long cnts[5] = {acc_n, acc_items, acc_ent, acc_ev, acc_cev};
        block_sum_multi<2, 5>(sums, cnts, s_red, s_redn);
        if (tid == 0) {
            const size_t o = ((size_t)ch * a.n_modes + ms) * N + q1;
            a.part_g[o] = sums[0];
            a.part_wp[o] = sums[1];
            a.part_n[o] = cnts[0];
            a.part_items[o] = cnts[1];
            a.part_ent[o] = cnts[2];
            if (a.part_ev) a.part_ev[o] = cnts[3];
            if (a.part_cev) a.part_cev[o] = cnts[4];
        }
    }
    if (dead && tid == 0) {
        // the abandoned units still get partial slots for the reduction to read (their Γ is
        // poisoned through the error flag)
        for (unit -= gridDim.x; unit < n_units; unit += gridDim.x) {
            const int ml = unit / N, q1 = unit - ml * N;
            const size_t o = ((size_t)ch * a.n_modes + mode0 + ml) * N + q1;
            a.part_g[o] = 0.0;
            a.part_wp[o] = 0.0;
            a.part_n[o] = 0;
            a.part_items[o] = 0;
            a.part_ent[o] = 0;
            if (a.part_ev) a.part_ev[o] = 0;
            if (a.part_cev) a.part_cev[o] = 0;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

template <bool ADA, int OP>
static cudaError_t launch_tc(const Tables &t, const RateArgs &a, int ch, int mode0, int nm, const float2 *w,
                             cudaStream_t s) {
    const size_t smem = tc_smem_bytes<OP>(t);
    cudaError_t e = cudaFuncSetAttribute(rates4_tc_kernel<ADA, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long units = (long long)nm * t.N;
    if (units > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>(units, (long long)std::max(sms, 1));   // one CTA per SM
    if (grid == 0) return cudaSuccess;
    rates4_tc_kernel<ADA, OP><<<grid, kTcThreads, smem, s>>>(t, a, ch, mode0, (int)units, w);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_tc_op(const Tables &t, const RateArgs &a, int ch, int mode0, int nm, const float2 *w,
                                cudaStream_t s) {
    return a.adaptive ? launch_tc<true, OP>(t, a, ch, mode0, nm, w, s) : launch_tc<false, OP>(t, a, ch, mode0, nm, w, s);
}

// Used for two-atom cells whose operands fit in shared memory in every format (other cells keep
// the CUDA-core kernels).
bool tc_supported(const Tables &t) {
    return t.n_atoms == 2 && tc_smem_bytes<kOpTF32x3>(t) <= 200 * 1024 && tc_smem_bytes<kOpF16x3>(t) <= 200 * 1024;
}

cudaError_t launch_rates4_tc(const Tables &t, const RateArgs &a, int ch, int mode0, int nm, const float2 *w,
                             cudaStream_t s) {
    if (t.n_atoms != 2) return cudaErrorInvalidValue;
    switch (a.use_tc) {
        case 1: return launch_tc_op<kOpF16x3>(t, a, ch, mode0, nm, w, s);
        case 2: return launch_tc_op<kOpBF16x3>(t, a, ch, mode0, nm, w, s);
        case 3: return launch_tc_op<kOpBF16>(t, a, ch, mode0, nm, w, s);
        case 4: return launch_tc_op<kOpTF32x3>(t, a, ch, mode0, nm, w, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
