// k_rates4_tc.cu - four-phonon +- channel, mixed precision, two-atom cells, with the cluster
// contraction X = Σ_r P_r^s2 W_r on the tensor cores (tcgen05).
//
// For a unit (λ, q') and a round of 128 partner points q'', the contraction of every (c, d) group
// of keys is a real matrix product per partner branch j':
//   [Xr | Xi](q'', γδ) = [Pr | s2 Pi](q'', r) . [[Wr, Wi], [-Wi, Wr]](r, γδ)
// (rows q'' = MMA M = 128 = TMEM lanes; K = 2 x keys of the group, padded to 16; N = 32 columns of
// which 18 hold the 9 complex γδ).  Operands are FP16 hi/lo splits (W scaled by a power of two
// per unit so that max |W| < 1), and three products hi.hi + hi.lo + lo.hi accumulate in FP32 in
// tensor memory: relative accuracy ~2^-21, the level of the FP32 CUDA-core contraction.  One
// elected thread issues tcgen05.mma (kind::f16) and tcgen05.commit to an mbarrier; every thread
// then reads its q'' row of X with tcgen05.ld.  The rows of partner points with kept processes
// are staged in shared memory and the compacted (q'', j') entries are evaluated exactly as in the
// CUDA-core tile kernel (Y = X e*''' per j''', V = e''.Y per kept j'', weights).
//
// Waits on the mbarrier are bounded (fc4_options.timeout_cycles SM clocks, default 2e9); on expiry the kernel
// sets the context's error flag (the reduction then writes NaN into Γ), waits once more (~1 s at
// most) for its MMAs in flight, frees its tensor memory and returns.
#include "k_rates4.cuh"

#include <cuda_fp16.h>

namespace fc4 {

namespace {

constexpr int kTcRows = 128;                // q'' per round = MMA M = TMEM lanes = threads
constexpr int kTcN = 32;                    // MMA N per (c, d) group (18 columns used)
constexpr int kTcCols = 128;                // TMEM columns: up to 4 groups x 32

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: canonical K-major layout without swizzle (8-row x 16-byte core
// matrices stored contiguously); lbo = byte step between core matrices along K, sbo = along M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major, M = 128, N = kTcN
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
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

__device__ __forceinline__ void split_f16(float x, __half &hi, __half &lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// byte offset of element (row, k) in a K-major no-swizzle FP16 tile with `rows` rows
__device__ __forceinline__ uint32_t tile_off(int row, int k, int rows) {
    return 128u * (uint32_t)((k >> 3) * (rows >> 3) + (row >> 3)) + 16u * (uint32_t)(row & 7) + 2u * (uint32_t)(k & 7);
}

}  // namespace

// Key layout of the contraction: group g = c NA + d holds keys [grp_start[g], grp_start[g+1]);
// its K extent is 2 x keys padded to 16 halves, at offset koff[g] (halves) of the K axis.
struct TcPlan {
    int kt;                   // total K (halves)
    int koff[4], kpad[4], nkey[4], r0[4];
};

template <int NA>
__host__ __device__ inline TcPlan tc_plan(const Tables &t) {
    TcPlan p{};
    int o = 0;
    for (int g = 0; g < NA * NA; ++g) {
        p.r0[g] = t.grp_start[g];
        p.nkey[g] = t.grp_start[g + 1] - t.grp_start[g];
        p.kpad[g] = (2 * p.nkey[g] + 15) / 16 * 16;
        p.koff[g] = o;
        o += p.kpad[g];
    }
    p.kt = o;
    return p;
}

// shared memory: A hi | A lo (128 x kt halves each) | B hi | B lo (32 x kt) | X rows | entries
template <int NA>
__host__ __device__ inline size_t tc_smem_bytes(const Tables &t) {
    const TcPlan p = tc_plan<NA>(t);
    return (size_t)2 * kTcRows * p.kt * 2 + (size_t)2 * kTcN * p.kt * 2 +
           (size_t)kTcRows * NA * NA * 9 * sizeof(float2) + (size_t)kTcRows * sizeof(unsigned long long) + 128;
}

template <int NA, bool ADA>
__global__ void __launch_bounds__(kTcRows, 2)
rates4_tc_kernel(const __grid_constant__ Tables t, const __grid_constant__ RateArgs a, int ch, int mode0,
                 const float2 *__restrict__ wall) {
    constexpr int NB = 3 * NA;
    constexpr int NG = NA * NA;
    const int s1 = (ch == 4) ? -1 : 1;
    const int s2 = (ch == 2) ? 1 : -1;
    const int N = t.N, nk = t.n_keys;
    const TcPlan pl = tc_plan<NA>(t);

    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *sA = tc_smem;                                            // hi, then lo at + 256 kt
    unsigned char *sB = sA + (size_t)2 * kTcRows * pl.kt * 2;            // hi, then lo at + 64 kt
    float2 *sX = reinterpret_cast<float2 *>(sB + (size_t)2 * kTcN * pl.kt * 2);   // [128][NG][9]
    unsigned long long *sE = reinterpret_cast<unsigned long long *>(sX + kTcRows * NG * 9);
    const uint32_t a_hi = smem_u32(sA), a_lo = a_hi + 256u * pl.kt;
    const uint32_t b_hi = smem_u32(sB), b_lo = b_hi + 64u * pl.kt;
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_scan[32];
    __shared__ double s_red[2 * 32];
    __shared__ long long s_redn[3 * 32];
    __shared__ float s_wmax[4];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int unit = blockIdx.x;
    const int ml = unit / N, q1 = unit - ml * N;
    const int ms = mode0 + ml;
    const int m0 = a.modes[ms];
    const int q0 = m0 / NB, j0 = m0 - q0 * NB;
    const float2 *ev = t.ev32;
    const float *occ = t.occ32;
    const float *invw = t.invw32;
    const long long spins = a.spin_limit > 0 ? a.spin_limit : 2000000000ll;   // ~1 s
    const uint32_t mbar = smem_u32(&s_mbar);

    Acc<float> acc_g, acc_wp;
    long long acc_n = 0, acc_items = 0, acc_ent = 0;
    const unsigned vm1 = t.vmask[q1];
    const bool active = !(q0 == 0 && j0 < 3) && vm1;

    if (active) {                                   // uniform across the block
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_u32(&s_tmem)), "r"(kTcCols));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        const float2 *wsrc = wall + (size_t)unit * (NB * nk * 9);
        // per-unit power-of-two scale of W: max |W| * 2^-E in [0.5, 1)
        float mx = 0.0f;
        for (int k = tid; k < NB * nk * 9; k += kTcRows) {
            const float2 w = wsrc[k];
            mx = fmaxf(mx, fmaxf(fabsf(w.x), fabsf(w.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
        if ((tid & 31) == 0) s_wmax[warp] = mx;
        // B padding (rows 18..31 and K columns beyond 2 x keys) is zero for the whole kernel
        for (int k = tid; k < 2 * kTcN * pl.kt / 2; k += kTcRows)
            reinterpret_cast<uint32_t *>(sB)[k] = 0u;
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t tmem = s_tmem;
        int e_w = 0;
        {
            const float m = fmaxf(fmaxf(s_wmax[0], s_wmax[1]), fmaxf(s_wmax[2], s_wmax[3]));
            if (m > 0.0f) frexpf(m, &e_w);
        }
        const float wscale = ldexpf(1.0f, -e_w), xscale = ldexpf(1.0f, e_w);

        const int4 c0 = t.qc[q0], c1 = t.qc[q1];
        const int b0 = c0.x + s1 * c1.x, b1 = c0.y + s1 * c1.y, b2 = c0.z + s1 * c1.z;
        const double w0 = t.om[m0];
        const float w0f = t.om32[m0];
        float base32[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) base32[j] = w0f + (float)s1 * t.om32[q1 * NB + j];
        uint32_t phase = 0;
        bool dead = false;

        for (int qb = 0; qb < N && !dead; qb += kTcRows) {
            const int q2 = qb + tid;
            const bool valid = q2 < N;
            int q3 = 0;
            // A row of this thread's q'': [Pr | s2 Pi] per group, FP16 hi / lo
            {
                const float2 *Prow = t.P4_32 + (size_t)(valid ? q2 : 0) * nk;
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    for (int k = 0; k < pl.kpad[g]; k += 2) {
                        float v[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int kk = k + u;
                            float x = 0.0f;
                            if (valid && kk < 2 * pl.nkey[g]) {
                                const float2 p = Prow[pl.r0[g] + (kk < pl.nkey[g] ? kk : kk - pl.nkey[g])];
                                x = kk < pl.nkey[g] ? p.x : (float)s2 * p.y;
                            }
                            v[u] = x;
                        }
                        __half h0, l0, h1, l1;
                        split_f16(v[0], h0, l0);
                        split_f16(v[1], h1, l1);
                        const uint32_t off = tile_off(tid, pl.koff[g] + k, kTcRows);
                        *reinterpret_cast<__half2 *>(sA + off) = __halves2half2(h0, h1);
                        *reinterpret_cast<__half2 *>(sA + 256u * pl.kt + off) = __halves2half2(l0, l1);
                    }
                }
            }
            // window: kept masks of this q'' for every partner branch j' (bit NB j''' + j'')
            unsigned long long keep[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) keep[j] = 0ull;
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
#pragma unroll
                for (int j1 = 0; j1 < NB; ++j1) {
                    if (!((vm1 >> j1) & 1u)) continue;
                    const float b = base32[j1];
                    if constexpr (ADA) {
                        unsigned long long kept = 0;
                        for (int j3 = 0; j3 < NB; ++j3)
                            if ((v3 >> j3) & 1u)
                                kept |= (unsigned long long)window_adaptive4_row<NB>(
                                            t, a, ch, s2, b, m0, q1 * NB + j1, q2, q3 * NB + j3, v2)
                                        << (NB * j3);
                        keep[j1] = kept;
                    } else {
                        unsigned long long sure = 0, amb = 0;
#pragma unroll
                        for (int j3 = 0; j3 < NB; ++j3)
#pragma unroll
                            for (int j2 = 0; j2 < NB; ++j2) {
                                const float ad = fabsf((b + w2f[j2]) - w3f[j3]);
                                const bool ok = ((v3 >> j3) & (v2 >> j2) & 1u) != 0;
                                sure |= (unsigned long long)(ok && ad <= a.lo32) << (NB * j3 + j2);
                                amb |= (unsigned long long)(ok && ad > a.lo32 && ad <= a.hi32) << (NB * j3 + j2);
                            }
                        while (amb) {
                            const int k = __ffsll(amb) - 1;
                            amb &= amb - 1;
                            const int j3 = k / NB, j2 = k - j3 * NB;
                            if (window_exact4(ch, w0, t.om[q1 * NB + j1], t.om[q2 * NB + j2], t.om[q3 * NB + j3],
                                              a.two_sigma))
                                sure |= 1ull << k;
                        }
                        keep[j1] = sure;
                    }
                }
            }

            for (int j1 = 0; j1 < NB && !dead; ++j1) {
                if (!((vm1 >> j1) & 1u)) continue;
                if (!__syncthreads_or(keep[j1] != 0ull)) continue;      // no entry in this round
                // B of (unit, j'): rows 2γδ (re) and 2γδ + 1 (im) of every group, FP16 hi / lo
                {
                    const float2 *wj = wsrc + (size_t)j1 * nk * 9;
                    for (int k = tid; k < nk * 9; k += kTcRows) {
                        const int r = k / 9, gd = k - r * 9;
                        int g = 0;
#pragma unroll
                        for (int gg = 1; gg < NG; ++gg) g += (r >= pl.r0[gg]);
                        const int kr = r - pl.r0[g];
                        const float2 w = wj[k];
                        const float wr = w.x * wscale, wi = w.y * wscale;
                        const float val[4] = {wr, -wi, wi, wr};    // (re row: k, K + k), (im row: k, K + k)
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int n = 2 * gd + (u >> 1);
                            const int kk = pl.koff[g] + kr + ((u & 1) ? pl.nkey[g] : 0);
                            __half h, l;
                            split_f16(val[u], h, l);
                            const uint32_t off = tile_off(n, kk, kTcN);
                            *reinterpret_cast<__half *>(sB + off) = h;
                            *reinterpret_cast<__half *>(sB + 64u * pl.kt + off) = l;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        for (int pz = 0; pz < 3; ++pz) {                 // hi.hi, hi.lo, lo.hi
                            const uint32_t ab = (pz == 2 ? a_lo : a_hi) + 256u * pl.koff[g];
                            const uint32_t bb = (pz == 1 ? b_lo : b_hi) + 64u * pl.koff[g];
                            for (int s = 0; s < pl.kpad[g] / 16; ++s)
                                mma_f16(tmem + (uint32_t)(kTcN * g), smem_desc(ab + 4096u * s, 2048u, 128u),
                                        smem_desc(bb + 1024u * s, 512u, 128u), (pz > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(mbar) : "memory");
                }
                const bool ok = mbar_wait(mbar, phase, spins);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {                             // the MMAs did not complete
                    if (tid == 0 && a.err) atomicExch(a.err, 1);
                    mbar_wait(mbar, phase ^ 1u, 2000000000ll);   // let the MMAs in flight finish
                    dead = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                // this thread's row of X (all groups), scaled back
                float xr[NG][18];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    if (pl.nkey[g] == 0) {
#pragma unroll
                        for (int k = 0; k < 18; ++k) xr[g][k] = 0.0f;
                    } else {
                        tmem_ld18(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kTcN * g), xr[g]);
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                // compact this j' 's entries; stage their X rows
                const unsigned long long mk = keep[j1];
                int total;
                const int off = block_exclusive_scan(mk != 0ull ? 1 : 0, s_scan, &total);
                if (mk) {
                    sE[off] = ((unsigned long long)tid << 48) | mk;
                    float2 *dst = sX + (size_t)off * NG * 9;
#pragma unroll
                    for (int g = 0; g < NG; ++g)
#pragma unroll
                        for (int k = 0; k < 9; ++k)
                            dst[g * 9 + k] = make_float2(xr[g][2 * k] * xscale, xr[g][2 * k + 1] * xscale);
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                for (int it = tid; it < total; it += kTcRows) {
                    ++acc_ent;
                    const unsigned long long e = sE[it];
                    const int iq2 = qb + (int)(e >> 48);
                    const int4 cc2 = t.qc[iq2];
                    const int iq3 = q_index_near(b0 + s2 * cc2.x, b1 + s2 * cc2.y, b2 + s2 * cc2.z,
                                                 t.mesh[0], t.mesh[1], t.mesh[2]);
                    const int m1 = q1 * NB + j1;
                    float ee1;
                    const float ex1 = two_sum(t.om32[m0], (float)s1 * t.om32[m1], ee1);
                    const float el01 = t.om32lo[m0] + (float)s1 * t.om32lo[m1];
                    const float iw01 = invw[m0] * invw[m1];
                    const float n1f = occ[m1];
                    float2 X[NA][NA][9];
                    const float2 *src = sX + (size_t)it * NG * 9;
#pragma unroll
                    for (int c = 0; c < NA; ++c)
#pragma unroll
                        for (int d = 0; d < NA; ++d)
#pragma unroll
                            for (int k = 0; k < 9; ++k) X[c][d][k] = src[(c * NA + d) * 9 + k];
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
                            acc_wp.add(w);
                            acc_g.add(w * (V.x * V.x + V.y * V.y));
                            acc_n += 1;
                        }
                    }
                }
                __syncthreads();                                         // sX / sE reused next
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
    }
    double sums[2] = {acc_g.value(), acc_wp.value()};
    long long cnts[3] = {acc_n, acc_items, acc_ent};
    block_sum_multi<2, 3>(sums, cnts, s_red, s_redn);
    if (threadIdx.x == 0) {
        const size_t o = ((size_t)ch * a.n_modes + ms) * N + q1;
        a.part_g[o] = sums[0];
        a.part_wp[o] = sums[1];
        a.part_n[o] = cnts[0];
        a.part_items[o] = cnts[1];
        a.part_ent[o] = cnts[2];
    }
}

template <int NA, bool ADA>
static cudaError_t launch_tc(const Tables &t, const RateArgs &a, int ch, int mode0, int nm, const float2 *w,
                             cudaStream_t s) {
    const size_t smem = tc_smem_bytes<NA>(t);
    cudaError_t e = cudaFuncSetAttribute(rates4_tc_kernel<NA, ADA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    rates4_tc_kernel<NA, ADA><<<(unsigned)((long long)nm * t.N), kTcRows, smem, s>>>(t, a, ch, mode0, w);
    return cudaGetLastError();
}

// Used for two-atom cells whose operands fit in shared memory next to a second block of the same
// size on the SM (other cells keep the CUDA-core kernels).
bool tc_supported(const Tables &t) {
    return t.n_atoms == 2 && tc_smem_bytes<2>(t) <= 110 * 1024;
}

cudaError_t launch_rates4_tc(const Tables &t, const RateArgs &a, int ch, int mode0, int nm, const float2 *w,
                             cudaStream_t s) {
    const bool ad = a.adaptive != 0;
    if (t.n_atoms != 2) return cudaErrorInvalidValue;
    return ad ? launch_tc<2, true>(t, a, ch, mode0, nm, w, s) : launch_tc<2, false>(t, a, ch, mode0, nm, w, s);
}

}  // namespace fc4
