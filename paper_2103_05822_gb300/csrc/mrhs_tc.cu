// Multi-right-hand-side aggregation / disaggregation on the tensor cores
// (tcgen05, sm_103a): the same chains as mrhs.cu (Figs. 2b, 3b with R columns),
// every step a grouped complex GEMM D = A B with FP32 accumulation in TMEM.
//
// Precision.  Each FP32 operand value v is split into T bfloat16 terms
// (T = 2: hi + lo, T = 3: hi + mid + lo; three terms represent an FP32 value
// exactly).  A product keeps the terms whose combined order is below T:
//   T = 2:  hi*hi + hi*lo + lo*hi
//   T = 3:  hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi
// and a complex product is four real ones,
//   Cr += Ar Br - Ai Bi,   Ci += Ar Bi + Ai Br,
// the minus sign taken by the MMA's negate-A bit.
//
// Layout.  An operand matrix is stored as 2T planes (re terms, then im terms)
// of bfloat16, "K-major": row = M (or N) index, K contiguous, leading dimension
// a multiple of 8 and zero beyond K.  A CTA computes a 128-row x BN tile
// (BN <= 128, multiple of 16); K goes in steps of 32 through a ring of shared
// memory stages filled by cp.async (zero-fill at ragged edges) in the
// no-swizzle canonical layout (8 x 16-byte core matrices; the next core matrix
// along K is 128 bytes on, the next 8 rows 512 bytes on).  One thread issues
// the MMAs of a stage and commits them to that stage's mbarrier, which frees
// the stage for the next load.  The epilogue reads Cr / Ci from TMEM (one row
// per thread) and writes the next step's operand planes, or the FP32 spectra /
// currents at the end of the chain.
//
// Steps (per group g and component alpha; see mrhs.cu for the FP32 version):
//   AG1  T^T (r_b x R)            = U_beta^T . X_g          A: U_beta^T [c][n]   B: X_g   [r][n]
//   AG2  M   (m x R)              = C_(3)^T  . T            A: C_(3)^T  [ab][c]  B: T     [r][c]
//        (the rows of C_(3)^T in the order b + r_p a, so that M' leaves in runs of b)
//   AG3  V'  (r_t R x n_phi)      = M'       . U_phi^T      A: M'  [a+r_t r][b]  B: U_phi [i_phi][b]
//   AG4  F'  (n_phi R x n_theta)  = V''      . U_theta^T    A: V'' [i_phi+n_phi r][a]  B: U_theta [i_theta][a]
//   DG1a P'  (n_phi R x r_t)      = G'       . U_theta      A: G'  [i_phi+n_phi r][i_theta]  B: U_theta^T [a][i_theta]
//   DG1b H'  (r_t R x r_p)        = P''      . U_phi        A: P'' [a+r_t r][i_phi]  B: U_phi^T [b][i_phi]
//   DG2  S   (r_b x R)            = C_(3)    . H            A: C_(3) [c][ab]  B: H [r][ab]
//   DG3  y_g (n_b x R)            = conj(U_beta^(0) S^(0) + U_beta^(1) S^(1))  A: U_beta [n][c]  B: S [r][c]
// The generic stage kernel (tc_gemm_kernel) runs these as listed.  Two kernels replace
// steps when the shapes allow: tc_ag34_kernel fuses AG3 and AG4 (V'' never leaves the
// SM), and tc_dg1a_kernel runs DG1a transposed, U_theta^T as A and 128 (i_phi, r)
// pairs of the spectra as N, so that its MMAs are wide.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <numeric>
#include <set>
#include <utility>
#include <vector>

#include "internal.h"

namespace tfmm {

namespace {

using bf16 = __nv_bfloat16;

constexpr int TBM = 128;       // MMA M
constexpr int TBK = 32;        // K per stage
constexpr int TBN_MAX = 128;   // largest BN
constexpr int TTHREADS = 128;  // 4 warps: one TMEM lane quarter each
constexpr int PLANE_TILE = 8192;  // bytes of one plane tile (128 rows x 32 K x 2 B)
constexpr long kWaitLimit = 1L << 26;

enum TcStage { TAG1, TAG2, TAG3, TAG4, TDG1A, TDG1B, TDG2, TDG3 };

struct TcCtx {
    const float2* spec_in;  // DG1a input (spectra; null: A from prepared planes)
    const float* w;         // DG1a quadrature weights (null: none)
    float2* spec;        // AG4 output (spectra)
    float2* y;           // DG3 output
    const int* grp_rwg;
    int64_t ld;          // ldy (DG3)
    float2 beta;         // DG3
    int R, G, n_theta, n_dir;
    int* err;            // set when a wait gives up
};

template <int T>
__host__ __device__ constexpr int n_products() { return T == 2 ? 3 : 6; }

// 32 consecutive TMEM columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t (&v)[32], uint32_t taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

// 8 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t (&v)[8], uint32_t taddr) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;   // next core matrix along K
    d |= (uint64_t)(512 >> 4) << 32;   // next 8-row group
    d |= (uint64_t)1 << 46;            // descriptor version (sm_100 family)
    return d;                          // base offset 0, no swizzle
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void cp16(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}

// v = t0 + t1 (+ t2) in bfloat16 terms, two values at once, one 32-bit word per term
// (x0's term in the low half, x1's in the high half): the hardware conversion rounds
// both to bfloat16 (to nearest, ties to even), the remainders are exact in FP32
// (within one bfloat16 unit of the value), and the same again.  Each remainder has at
// most 16, then 8 significant bits, so three terms hold every FP32 value exactly (down
// to where the remainders become FP32 subnormals, below about 1e-30).  Rounding to
// nearest is odd in its argument: the terms of -x are the terms of x, negated.
template <int T>
__device__ __forceinline__ void split_pack(float x0, float x1, uint32_t (&w)[3]) {
    uint32_t h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
    w[0] = h;
    const float r0 = x0 - __uint_as_float(h << 16), r1 = x1 - __uint_as_float(h & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(r1), "f"(r0));
    w[1] = h;
    if (T == 3) {
        const float s0 = r0 - __uint_as_float(h << 16), s1 = r1 - __uint_as_float(h & 0xffff0000u);
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(s1), "f"(s0));
        w[2] = h;
    }
}

template <int T>
__device__ __forceinline__ void store_planes(bf16* base, int64_t ps, int64_t idx, float2 v) {
    uint32_t w[3];
    split_pack<T>(v.x, v.y, w);  // term p of the real part in the low half, of the imaginary part in the high
#pragma unroll
    for (int p = 0; p < T; ++p) {
        base[p * ps + idx] = __ushort_as_bfloat16((unsigned short)(w[p] & 0xffffu));
        base[(T + p) * ps + idx] = __ushort_as_bfloat16((unsigned short)(w[p] >> 16));
    }
}

// DG1a A operand straight from the FP32 spectra: row m = i_phi + n_phi r, depth
// i_theta; each element conj(W g) (Fig. 3b step 1 with the quadrature weights),
// split into BF16 terms in registers.  Plain loads: the data pass through once.
template <int T>
__device__ __forceinline__ void load_g_tile(uint8_t* st, const TcCtx& c, const TcProb& p, int m0, int k0) {
    constexpr int ITER = TBM * 4 / TTHREADS;
    const int nt = c.n_theta;
    float2 v[ITER][8];
    // every load of this thread first (memory-level parallelism), then the splits
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int idx = threadIdx.x + i * TTHREADS, r = idx >> 2, kc = idx & 3;
        const int m = m0 + r, k = k0 + kc * 8;
        const bool row_ok = m < p.M;
        const int ip = row_ok ? m % p.n_phi : 0, rr = row_ok ? m / p.n_phi : 0;
        const int64_t o = (((int64_t)rr * c.G + p.g) * 2 + p.alpha) * c.n_dir + (int64_t)nt * ip;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int th = k + e;
            v[i][e] = make_float2(0.f, 0.f);
            if (row_ok && th < nt) {
                const float2 g = __ldg(c.spec_in + o + th);
                const float wt = c.w ? __ldg(c.w + th + (int64_t)nt * ip) : 1.0f;
                v[i][e] = make_float2(wt * g.x, -wt * g.y);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int idx = threadIdx.x + i * TTHREADS, r = idx >> 2, kc = idx & 3;
        uint32_t w[2 * T][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint32_t pr[3], pi[3];
            split_pack<T>(v[i][e].x, v[i][e + 1].x, pr);
            split_pack<T>(v[i][e].y, v[i][e + 1].y, pi);
#pragma unroll
            for (int q = 0; q < T; ++q) {
                w[q][e / 2] = pr[q];
                w[T + q][e / 2] = pi[q];
            }
        }
        const int off = (r >> 3) * 512 + kc * 128 + (r & 7) * 16;
#pragma unroll
        for (int q = 0; q < 2 * T; ++q)
            *reinterpret_cast<uint4*>(st + q * PLANE_TILE + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

// Loads k-tile `kt` of the problem's A (128 rows from m0) and B (BN rows from n0) into one
// stage, NTHR threads sharing the copies.
template <int T, int S, int NTHR = TTHREADS>
__device__ __forceinline__ void load_stage(uint8_t* st, const TcCtx& c, const TcProb& p, int m0, int n0, int kt,
                                           int kt0) {
    const bool seg1 = kt >= kt0;
    const int k0 = (seg1 ? kt - kt0 : kt) * TBK;
    const int K = seg1 ? p.K1 : p.K0;
    const int K8 = (K + 7) & ~7;
    const bf16* A = seg1 ? p.A1 : p.A0;
    const bf16* B = seg1 ? p.B1 : p.B0;
    const int64_t ald = seg1 ? p.a_ld1 : p.a_ld0, aps = seg1 ? p.a_ps1 : p.a_ps0;
    const int64_t bld = seg1 ? p.b_ld1 : p.b_ld0, bps = seg1 ? p.b_ps1 : p.b_ps0;
    const int na = (S == TDG1A && c.spec_in) ? 0 : 2 * T * TBM * 4;
    if constexpr (S == TDG1A) {
        static_assert(NTHR == TTHREADS, "the spectra tile loader assumes one 128-thread CTA");
        if (c.spec_in) load_g_tile<T>(st, c, p, m0, k0);
    }
    for (int idx = threadIdx.x; idx < na; idx += NTHR) {
        const int pl = idx / (TBM * 4), rem = idx % (TBM * 4), r = rem >> 2, kc = rem & 3;
        const int m = m0 + r, k = k0 + kc * 8;
        const bool ok = m < p.M && k < K8;
        const bf16* src = ok ? A + pl * aps + (int64_t)m * ald + k : A;
        cp16(st + pl * PLANE_TILE + (r >> 3) * 512 + kc * 128 + (r & 7) * 16, src, ok ? 16 : 0);
    }
    const int nb = 2 * T * p.BN * 4;
    uint8_t* sb = st + 2 * T * PLANE_TILE;
    for (int idx = threadIdx.x; idx < nb; idx += NTHR) {
        const int pl = idx / (p.BN * 4), rem = idx % (p.BN * 4), r = rem >> 2, kc = rem & 3;
        const int n = n0 + r, k = k0 + kc * 8;
        const bool ok = n < p.N && k < K8;
        const bf16* src = ok ? B + pl * bps + (int64_t)n * bld + k : B;
        cp16(sb + pl * PLANE_TILE + (r >> 3) * 512 + kc * 128 + (r & 7) * 16, src, ok ? 16 : 0);
    }
}

template <int T, int S>
__device__ __forceinline__ void epilogue(const TcCtx& c, const TcProb& p, int i, int j, float2 v) {
    bf16* o = reinterpret_cast<bf16*>(p.out);
    switch (S) {
        case TAG1:  // T stored [r][c]: row j (= r), column i (= c)
            store_planes<T>(o, p.o_ps, (int64_t)j * p.o_ld + i, v);
            break;
        case TAG2: {  // M' stored [a + r_t r][b]; i = b + r_p a (the order of the C_(3)^T planes), j = r
            const int rp = p.M / p.rt, a = i / rp, b = i % rp;
            store_planes<T>(o, p.o_ps, (int64_t)(a + p.rt * j) * p.o_ld + b, v);
        } break;
        case TAG3: {  // V'' stored [i_phi + n_phi r][a]; i = a + r_t r, j = i_phi
            const int a = i % p.rt, r = i / p.rt;
            store_planes<T>(o, p.o_ps, (int64_t)(j + p.n_phi * r) * p.o_ld + a, v);
        } break;
        case TAG4: {  // spectra; i = i_phi + n_phi r, j = i_theta
            const int ip = i % p.n_phi, r = i / p.n_phi;
            float2* F = c.spec;
            F[(((int64_t)r * c.G + p.g) * 2 + p.alpha) * c.n_dir + j + (int64_t)c.n_theta * ip] = v;
        } break;
        case TDG1A: {  // P'' stored [a + r_t r][i_phi]; i = i_phi + n_phi r, j = a
            const int ip = i % p.n_phi, r = i / p.n_phi;
            store_planes<T>(o, p.o_ps, (int64_t)(j + p.rt * r) * p.o_ld + ip, v);
        } break;
        case TDG1B: {  // H stored [r][a + r_t b]; i = a + r_t r, j = b
            const int a = i % p.rt, r = i / p.rt;
            store_planes<T>(o, p.o_ps, (int64_t)r * p.o_ld + a + p.rt * j, v);
        } break;
        case TDG2:  // S stored [r][c]; i = c, j = r
            store_planes<T>(o, p.o_ps, (int64_t)j * p.o_ld + i, v);
            break;
        case TDG3: {  // y = beta y + conj(v); i = n, j = r
            float2* dst = c.y + (int64_t)c.grp_rwg[p.rwg + i] + c.ld * j;
            float2 r = make_float2(v.x, -v.y);
            if (c.beta.x != 0.f || c.beta.y != 0.f) {
                const float2 old = *dst;
                r.x += c.beta.x * old.x - c.beta.y * old.y;
                r.y += c.beta.x * old.y + c.beta.y * old.x;
            }
            *dst = r;
        } break;
    }
}

// Adds 64 columns (from col) of the accumulator pair at TMEM column `base` (re) and
// base + cofs (im) of this warp's lane quarter into registers; columns past bn skipped.
__device__ __forceinline__ void drain_add(float (&ar)[64], float (&ai)[64], uint32_t base, int cofs, int col,
                                          int bn) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
        if (col + c0 < bn) {  // warp-uniform
            uint32_t vr[32], vi[32];
            tmem_ld32(vr, base + col + c0);
            tmem_ld32(vi, base + cofs + col + c0);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                ar[c0 + j] += __uint_as_float(vr[j]);
                ai[c0 + j] += __uint_as_float(vi[j]);
            }
        }
    }
}

// nst: stages of the shared-memory ring (1 .. NST_MAX); tcols: TMEM columns allocated
// (Cr at column 0, Ci at column cofs).
//
// CH (chunked accumulation, needs hsplit): the accumulation in TMEM rounds toward
// zero at every MMA, so its error grows with the number of K steps summed into one
// accumulator.  With CH the leading products (hi x hi) start a fresh accumulator
// every `chunk` k-tiles; at the end of each chunk the CTA waits for its MMAs and
// adds the accumulator into FP32 registers (round to nearest), so no accumulator
// sees more than 2 chunk K steps of 16.  The correction products, 2^-8 smaller,
// stay in one accumulator over the whole K.  Eight warps: warps w and w + 4 read
// lane quarter w & 3 of TMEM and hold 64 columns each.
template <int T, int S, bool CH>
__global__ void __launch_bounds__(CH ? 2 * TTHREADS : TTHREADS)
    tc_gemm_kernel(const TcCtx c, const TcProb* __restrict__ probs, const MrTile* __restrict__ tiles, int nst,
                   int tcols, int cofs, int hsplit, int chunk) {
    constexpr int NST_MAX = (T == 2) ? 3 : 2;
    constexpr int STAGE = 2 * 2 * T * PLANE_TILE;
    constexpr int NTHR = CH ? 2 * TTHREADS : TTHREADS;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar[NST_MAX];
    __shared__ uint32_t tmem_base;
    const int NST = nst;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const MrTile t = tiles[blockIdx.x];
    const TcProb p = probs[t.prob];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0)
        for (int s = 0; s < NST; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[s])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = tmem_base;
    const int kt0 = (p.K0 + TBK - 1) / TBK;
    const int KT = kt0 + (p.K1 > 0 ? (p.K1 + TBK - 1) / TBK : 0);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(p.BN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
    const uint32_t idesc_neg = idesc | (1u << 13);
    // CH: this warp's TMEM lanes and 64 columns, and their running FP32 sums
    const uint32_t q_lanes = (uint32_t)((warp & 3) * 32) << 16;
    const int q_col = (warp >> 2) * 64;
    float accr[CH ? 64 : 1], acci[CH ? 64 : 1];
    if constexpr (CH) {
#pragma unroll
        for (int j = 0; j < 64; ++j) accr[j] = acci[j] = 0.f;
    }
    bool ok = true;
    // prologue: k-tiles 0 .. NST-2
    for (int s = 0; s < NST - 1; ++s) {
        if (s < KT) load_stage<T, S, NTHR>(smem + s * STAGE, c, p, t.m0, t.n0, s, kt0);
        asm volatile("cp.async.commit_group;");
    }
    (void)STAGE;
    for (int kt = 0; kt < KT; ++kt) {
        const int b = kt % NST;
        if (NST == 1) {  // single buffer: reload it once the previous k-tile's MMAs are done
            if (kt >= 1) ok = ok && mbar_wait(&mbar[0], (kt - 1) & 1);
            if (ok) load_stage<T, S, NTHR>(smem, c, p, t.m0, t.n0, kt, kt0);
            asm volatile("cp.async.commit_group;");
            asm volatile("cp.async.wait_group 0;");
        } else if (NST == 2) {
            asm volatile("cp.async.wait_group 0;");
        } else {
            asm volatile("cp.async.wait_group 1;");
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = smem_u32(smem + b * STAGE);
            constexpr int PI[6] = {0, 0, 1, 0, 1, 2}, PJ[6] = {0, 1, 0, 2, 1, 0};
            // K steps of 16 that hold data in this k-tile (the zero tail past K is skipped)
            const int kseg = kt >= kt0 ? p.K1 : p.K0, koff = (kt >= kt0 ? kt - kt0 : kt) * TBK;
            const int nsteps = min(2, (kseg - koff + 15) / 16);
            const bool fresh = CH && (kt % chunk) == 0;  // first k-tile of a chunk
#pragma unroll
            for (int s16 = 0; s16 < 2; ++s16)
#pragma unroll
                for (int q = 0; q < n_products<T>(); ++q) {
                    if (s16 >= nsteps) break;
                    const uint32_t ar = base + PI[q] * PLANE_TILE + s16 * 256;
                    const uint32_t ai = base + (T + PI[q]) * PLANE_TILE + s16 * 256;
                    const uint32_t br = base + (2 * T + PJ[q]) * PLANE_TILE + s16 * 256;
                    const uint32_t bi = base + (2 * T + T + PJ[q]) * PLANE_TILE + s16 * 256;
                    // hsplit: the leading product (hi x hi) and the correction products
                    // accumulate apart (columns 0 / 2 cofs), summed in FP32 by the epilogue
                    const bool lo = hsplit && q > 0;
                    uint32_t acc = (kt > 0 || s16 > 0 || q > (lo ? 1 : 0) || (q > 0 && !hsplit)) ? 1u : 0u;
                    if (CH && !lo) acc = (fresh && s16 == 0) ? 0u : 1u;
                    const uint32_t d = tm + (lo ? 2 * cofs : 0);
                    mma_bf16(d, make_desc(ar), make_desc(br), idesc, acc);
                    mma_bf16(d, make_desc(ai), make_desc(bi), idesc_neg, 1u);
                    mma_bf16(d + cofs, make_desc(ar), make_desc(bi), idesc, acc);
                    mma_bf16(d + cofs, make_desc(ai), make_desc(br), idesc, 1u);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[b])));
        }
        // refill the stage that k-tile kt - 1 used, once its MMAs are done
        if (NST > 1) {
            const int nk = kt + NST - 1;
            if (nk < KT) {
                if (kt >= 1) ok = ok && mbar_wait(&mbar[(kt - 1) % NST], ((kt - 1) / NST) & 1);
                if (ok) load_stage<T, S, NTHR>(smem + (nk % NST) * STAGE, c, p, t.m0, t.n0, nk, kt0);
            }
            asm volatile("cp.async.commit_group;");
        }
        if constexpr (CH) {
            if (kt % chunk == chunk - 1 && kt + 1 < KT) {
                // end of a chunk: once its MMAs are done, add the leading-product
                // accumulator into the registers; the next k-tile restarts it
                ok = mbar_wait(&mbar[b], (kt / NST) & 1) && ok;
                ok = __syncthreads_and(ok);
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (ok) drain_add(accr, acci, tm + q_lanes, cofs, q_col, p.BN);
                asm volatile("tcgen05.fence::before_thread_sync;");
            }
        }
    }
    asm volatile("cp.async.wait_group 0;");
    // always wait (bounded) for the last commit: no MMA may still read TMEM when it is freed
    if (KT > 0 && !mbar_wait(&mbar[(KT - 1) % NST], ((KT - 1) / NST) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // one outcome for the whole CTA: the TMEM loads below are warp-collective
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicAdd(c.err, 1);
    } else if constexpr (CH) {
        // the last chunk and the correction products, then the outputs from registers
        drain_add(accr, acci, tm + q_lanes, cofs, q_col, p.BN);
        drain_add(accr, acci, tm + q_lanes + 2 * cofs, cofs, q_col, p.BN);
        const int row = t.m0 + (warp & 3) * 32 + lane;
        if (row < p.M) {
#pragma unroll
            for (int jj = 0; jj < 64; ++jj) {
                const int cc = q_col + jj, col = t.n0 + cc;
                if (cc < p.BN && col < p.N) epilogue<T, S>(c, p, row, col, make_float2(accr[jj], acci[jj]));
            }
        }
    } else {
        const int row = t.m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < p.BN; c0 += 32) {
            uint32_t vr[32], vi[32];
            const uint32_t ta = tm + ((uint32_t)(warp * 32) << 16) + c0;
            tmem_ld32(vr, ta);
            tmem_ld32(vi, ta + cofs);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (hsplit) {
                uint32_t w[32];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    tmem_ld32(w, ta + 2 * cofs + h * cofs);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    uint32_t* v = h ? vi : vr;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) v[jj] = __float_as_uint(__uint_as_float(v[jj]) + __uint_as_float(w[jj]));
                }
            }
            if (row < p.M) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int col = t.n0 + c0 + jj;
                    if (c0 + jj < p.BN && col < p.N)
                        epilogue<T, S>(c, p, row, col, make_float2(__uint_as_float(vr[jj]), __uint_as_float(vi[jj])));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tcols));
}

// ------------------------------------------------------ fused AG3 + AG4
// One CTA per (item, block of nr RHS).  AG3 runs as one GEMM with the phi
// directions on the TMEM lanes, D1[i_phi][(a, r)] = sum_b U_phi[i_phi][b] M'_r[a][b]
// (Fig. 2b step 2); then for each r of the block V_r = D1[:, (., r)] goes
// TMEM -> registers -> shared memory (split into BF16 terms) as the A operand of
// AG4, F_r[i_phi][i_theta] = sum_a V_r[i_phi][a] U_theta[i_theta][a] (Fig. 2b
// steps 3-4), which leaves TMEM straight for the spectra.  The MMAs of r overlap
// the spectra stores of r - 1 (two D2 accumulators).
struct F34Item {
    const bf16* uph; int64_t uph_ld, uph_ps;  // U_phi planes [i_phi][b]
    const bf16* uth; int64_t uth_ld, uth_ps;  // U_theta planes [i_theta][a]
    const bf16* m;   int64_t m_ld, m_ps;      // M' planes [a + r_t r][b]
    int g, alpha, rt, rp;
};
struct F34Tile { int item, r0, nr; };

__device__ __forceinline__ uint64_t make_desc_sbo(uint32_t addr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;              // next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;   // next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}

// 2T planes of `rows` rows (zero-filled from row `valid` and from column r8(kvalid))
// of a K-major source into the canonical no-swizzle layout with depth K.
template <int T>
__device__ __forceinline__ void load_planes(uint8_t* dst, int plane_bytes, int K, const bf16* src, int64_t ld,
                                            int64_t ps, int rows, int valid, int kvalid) {
    const int kc8 = K / 8, k8v = (kvalid + 7) / 8;
    const int total = 2 * T * rows * kc8;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int pl = idx / (rows * kc8), rem = idx % (rows * kc8), r = rem / kc8, kc = rem % kc8;
        const bool ok = r < valid && kc < k8v;
        const bf16* g = ok ? src + pl * ps + (int64_t)r * ld + kc * 8 : src;
        cp16(dst + pl * plane_bytes + (r >> 3) * (K * 16) + kc * 128 + (r & 7) * 16, g, ok ? 16 : 0);
    }
}

// The accumulation in TMEM rounds toward zero at every MMA, relative to the
// accumulator's current magnitude.  With the whole K in shared memory, the kernels
// below issue every correction product (2^-8 smaller than the leading hi x hi
// product) over all K steps first, while the accumulator is still small, and the
// leading products last: the leading accumulation then sees only 2 MMAs per K step
// at full scale, as with a separate accumulator, without its TMEM columns.
template <int T>
__device__ __forceinline__ int product_order(int i) {  // corrections first, hi x hi last
    return i + 1 < n_products<T>() ? i + 1 : 0;
}

template <int T>
__device__ __forceinline__ void issue_products(uint32_t d_re, uint32_t d_im, uint32_t a, int a_plane, uint32_t b,
                                               int b_plane, uint32_t sbo_a, uint32_t sbo_b, int ksteps,
                                               uint32_t idesc) {
    constexpr int PI[6] = {0, 0, 1, 0, 1, 2}, PJ[6] = {0, 1, 0, 2, 1, 0};
    const uint32_t idesc_neg = idesc | (1u << 13);
    // the start-address field holds addr >> 4 (shared memory < 256 KB): offsets add to it
    const uint64_t da = make_desc_sbo(a, sbo_a), db = make_desc_sbo(b, sbo_b);
    const uint32_t ta = (uint32_t)T * a_plane >> 4, tb = (uint32_t)T * b_plane >> 4;
#pragma unroll
    for (int i = 0; i < n_products<T>(); ++i) {
        const int q = product_order<T>(i);
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t ar = da + (uint32_t)(PI[q] * a_plane + ks * 256) / 16, ai = ar + ta;
            const uint64_t br = db + (uint32_t)(PJ[q] * b_plane + ks * 256) / 16, bi = br + tb;
            const uint32_t acc = (ks > 0 || i > 0) ? 1u : 0u;
            mma_bf16(d_re, ar, br, idesc, acc);
            mma_bf16(d_re, ai, bi, idesc_neg, 1u);
            mma_bf16(d_im, ar, bi, idesc, acc);
            mma_bf16(d_im, ai, br, idesc, 1u);
        }
    }
}

// Complex products with the real and imaginary parts side by side in an
// accumulator of 2N columns: B holds per term q three planes of N rows,
// (-Im_q, Re_q, Im_q), so rows [Re_q; Im_q] and [-Im_q; Re_q] are each one
// 2N-row operand.  d0 += Ar [Br | Bi], d1 += Ai [-Bi | Br]; d0 + d1 is the
// product (d1 may equal d0).
template <int T>
__device__ __forceinline__ void issue_products_cat(uint32_t d0, uint32_t d1, uint32_t a, int a_plane, uint32_t b,
                                                   int b_slot, uint32_t sbo_a, uint32_t sbo_b, int ksteps,
                                                   uint32_t idesc) {
    constexpr int PI[6] = {0, 0, 1, 0, 1, 2}, PJ[6] = {0, 1, 0, 2, 1, 0};
    const uint64_t da = make_desc_sbo(a, sbo_a), db = make_desc_sbo(b, sbo_b);
    const uint32_t ta = (uint32_t)T * a_plane >> 4;
#pragma unroll
    for (int i = 0; i < n_products<T>(); ++i) {  // corrections first, hi x hi last (see issue_products)
        const int q = product_order<T>(i);
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t ar = da + (uint32_t)(PI[q] * a_plane + ks * 256) / 16, ai = ar + ta;
            const uint64_t bneg = db + (uint32_t)(3 * PJ[q] * b_slot + ks * 256) / 16, bpos = bneg + b_slot / 16;
            const uint32_t acc = (ks > 0 || i > 0) ? 1u : 0u;
            mma_bf16(d0, ar, bpos, idesc, acc);
            mma_bf16(d1, ai, bneg, idesc, d1 == d0 ? 1u : acc);
        }
    }
}

__device__ __forceinline__ uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

// ------------------------------------------- stage kernel with a TMA-fed ring
// The long-K stages (AG1, AG2, DG2, DG3) as tc_gemm_kernel<T, S, true>, the same MMAs in
// the same order and the same chunked accumulation, but with the operands fed by the
// tensor-memory accelerator: one thread keeps `nst` K steps of 16 in flight (two 3-D
// boxes of 8 K x rows x 2T planes per operand and K step, zero-filled past the matrix
// edges by the copy engine), issues the MMAs of a K step as soon as its bytes have
// arrived and refills the stage of the previous K step once those MMAs are done; the
// other threads only take part in the chunk drains and the epilogue.  A box lands in
// shared memory as [8-element K chunk][plane][row][8 elements], i.e. 8 x 16-byte core
// matrices with the next 8 rows 128 bytes on and the next K chunk one box on, which is
// what the MMA descriptors below describe.
constexpr int NST_TMA_MAX = 8;

__device__ __forceinline__ uint64_t make_desc_lbo(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;   // next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;   // next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int T, int S>
__global__ void __launch_bounds__(2 * TTHREADS)
    tc_gemm_tma_kernel(const TcCtx c, const TcProb* __restrict__ probs, const CUtensorMap* __restrict__ maps,
                       const MrTile* __restrict__ tiles, int nst, int tcols, int cofs, int chunk) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[NST_TMA_MAX], empty[NST_TMA_MAX];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const MrTile t = tiles[blockIdx.x];
    const TcProb p = probs[t.prob];
    const CUtensorMap* mp = maps + 4 * (int64_t)t.prob;  // A0, B0, A1, B1
    const int BN = p.BN;
    const int abox = 8 * TBM * 2 * T * 2, bbox = 8 * BN * 2 * T * 2;
    const int stage_bytes = 2 * abox + 2 * bbox;  // one K step of 16
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0)
        for (int s = 0; s < nst; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(1));
        }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = tmem_base;
    const int ks0 = (p.K0 + 15) / 16, kt0 = (p.K0 + 31) / 32;
    const int KS = ks0 + (p.K1 > 0 ? (p.K1 + 15) / 16 : 0);
    // chunks of `chunk` k-tiles of 32 as in tc_gemm_kernel (a segment's last k-tile may hold
    // one K step), so that both kernels round alike: k-tile of a K step, and its first / last
    auto ktile = [&](int ks) { return ks < ks0 ? ks / 2 : kt0 + (ks - ks0) / 2; };
    auto kt_first = [&](int ks) { return ks < ks0 ? (ks % 2) == 0 : ((ks - ks0) % 2) == 0; };
    auto kt_last = [&](int ks) { return ks + 1 == KS || ks + 1 == ks0 || ktile(ks + 1) != ktile(ks); };
    auto produce = [&](int ks) {
        uint8_t* base = smem + (ks % nst) * stage_bytes;
        const bool seg1 = ks >= ks0;
        const int koff = (seg1 ? ks - ks0 : ks) * 16;
        const CUtensorMap* ma = mp + (seg1 ? 2 : 0);
        const CUtensorMap* mb = mp + (seg1 ? 3 : 1);
        uint64_t* bar = &full[ks % nst];
        mbar_expect_tx(bar, (uint32_t)stage_bytes);
        tma_load_3d(base, ma, koff, t.m0, 0, bar);
        tma_load_3d(base + abox, ma, koff + 8, t.m0, 0, bar);
        tma_load_3d(base + 2 * abox, mb, koff, t.n0, 0, bar);
        tma_load_3d(base + 2 * abox + bbox, mb, koff + 8, t.n0, 0, bar);
    };
    int produced = 0, consumed = 0;
    if (tid == 0)
        for (; produced < min(nst, KS); ++produced) produce(produced);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
    const uint32_t idesc_neg = idesc | (1u << 13);
    const uint32_t q_lanes = (uint32_t)((warp & 3) * 32) << 16;
    const int q_col = (warp >> 2) * 64;
    float accr[64], acci[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) accr[j] = acci[j] = 0.f;
    bool ok = true;
    for (int ks = 0; ks < KS; ++ks) {
        const int st = ks % nst;
        const uint32_t ph = (uint32_t)(ks / nst) & 1u;
        if (tid == 0 && ok) {
            ok = mbar_wait(&full[st], ph);
            if (ok) {
                consumed = ks + 1;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t base = smem_u32(smem + st * stage_bytes);
                constexpr int PI[6] = {0, 0, 1, 0, 1, 2}, PJ[6] = {0, 1, 0, 2, 1, 0};
                const bool fresh = (ktile(ks) % chunk) == 0 && kt_first(ks);  // first K step of a chunk
#pragma unroll
                for (int q = 0; q < n_products<T>(); ++q) {
                    const uint64_t ar = make_desc_lbo(base + PI[q] * TBM * 16, abox, 128);
                    const uint64_t ai = make_desc_lbo(base + (T + PI[q]) * TBM * 16, abox, 128);
                    const uint64_t br = make_desc_lbo(base + 2 * abox + PJ[q] * BN * 16, bbox, 128);
                    const uint64_t bi = make_desc_lbo(base + 2 * abox + (T + PJ[q]) * BN * 16, bbox, 128);
                    // the leading product (hi x hi) restarts its accumulator every chunk; the
                    // correction products accumulate apart over the whole K (columns 2 cofs on)
                    const bool lo = q > 0;
                    const uint32_t acc = lo ? ((ks > 0 || q > 1) ? 1u : 0u) : (fresh ? 0u : 1u);
                    const uint32_t d = tm + (lo ? 2 * cofs : 0);
                    mma_bf16(d, ar, br, idesc, acc);
                    mma_bf16(d, ai, bi, idesc_neg, 1u);
                    mma_bf16(d + cofs, ar, bi, idesc, acc);
                    mma_bf16(d + cofs, ai, br, idesc, 1u);
                }
                mma_commit(&empty[st]);
                // refill the stage of K step ks - 1 once its MMAs are done (those of ks keep
                // the tensor pipe busy meanwhile)
                if (ks >= 1 && produced < KS) {
                    ok = mbar_wait(&empty[(ks - 1) % nst], (uint32_t)((ks - 1) / nst) & 1u);
                    if (ok) produce(produced++);
                }
            }
        }
        if (kt_last(ks) && (ktile(ks) % chunk) == chunk - 1 && ks + 1 < KS) {
            // end of a chunk: once its MMAs are done, add the leading-product accumulator
            // into the registers; the next K step restarts it
            ok = mbar_wait(&empty[st], ph) && ok;
            ok = __syncthreads_and(ok);
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (ok) drain_add(accr, acci, tm + q_lanes, cofs, q_col, BN);
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }
    // always wait (bounded) for the last commit: no MMA may still read TMEM when it is freed
    if (KS > 0 && !mbar_wait(&empty[(KS - 1) % nst], (uint32_t)((KS - 1) / nst) & 1u)) ok = false;
    if (tid == 0)  // copies still in flight after a wait gave up land before the CTA exits
        for (int ks = consumed; ks < produced; ++ks) mbar_wait(&full[ks % nst], (uint32_t)(ks / nst) & 1u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicAdd(c.err, 1);
    } else {
        drain_add(accr, acci, tm + q_lanes, cofs, q_col, BN);
        drain_add(accr, acci, tm + q_lanes + 2 * cofs, cofs, q_col, BN);
        const int row = t.m0 + (warp & 3) * 32 + lane;
        if (row < p.M) {
#pragma unroll
            for (int jj = 0; jj < 64; ++jj) {
                const int cc = q_col + jj, col = t.n0 + cc;
                if (cc < BN && col < p.N) epilogue<T, S>(c, p, row, col, make_float2(accr[jj], acci[jj]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tcols));
}

constexpr int F34_WORKERS = 512;               // 16 warps, four per TMEM lane quarter
constexpr int F34_THREADS = F34_WORKERS + 32;  // and one warp that only issues MMAs

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void workers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(F34_WORKERS) : "memory");
}

// mbarriers of the fused kernel
enum { F34_D1 = 0, F34_A2 = 1, F34_D2 = 3, F34_EMPTY = 5, F34_NBAR = 7 };

template <int T>
__global__ void __launch_bounds__(F34_THREADS) tc_ag34_kernel(const TcCtx c, const F34Item* __restrict__ items,
                                                             const F34Tile* __restrict__ tiles, const FusedShape sh,
                                                             int n_phi) {
    extern __shared__ __align__(1024) uint8_t smem[];
    // F34_D1: AG3 done; F34_A2 + b: A2[b] written; F34_D2 + b: AG4 into D2[b] done;
    // F34_EMPTY + b: D2[b] read out
    __shared__ __align__(8) uint64_t mbar[F34_NBAR];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const F34Tile t = tiles[blockIdx.x];
    const F34Item it = items[t.item];
    const int K1 = sh.K1, K2 = sh.K2, nt = c.n_theta;
    const int a1p = TBM * K1 * 2, b1p = sh.N1p * K1 * 2, b2p = sh.ntp * K2 * 2, a2p = TBM * K2 * 2;
    // U_phi and M' are dead once AG3 is done: the spectra staging reuses the first,
    // the two A operands of AG4 the second
    const int r1 = max(2 * T * a1p, n_phi * nt * 8), r2 = max(2 * T * b1p, 2 * 2 * T * a2p);
    uint8_t* sA1 = smem;
    float2* stage = reinterpret_cast<float2*>(smem);
    uint8_t* sB1 = smem + r1;
    uint8_t* sA2b = sB1;
    uint8_t* sB2 = sB1 + r2;  // 3T slots (-Im_q, Re_q, Im_q) of b2p bytes
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(sh.tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0)
        for (int b = 0; b < F34_NBAR; ++b) {
            const int cnt = (b == F34_A2 || b == F34_A2 + 1 || b == F34_EMPTY || b == F34_EMPTY + 1) ? F34_WORKERS : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[b])), "r"(cnt));
        }
    asm volatile("fence.mbarrier_init.release.cluster;");
    const int n1 = it.rt * t.nr, n1p = (n1 + 15) & ~15;
    load_planes<T>(sA1, a1p, K1, it.uph, it.uph_ld, it.uph_ps, n_phi, n_phi, it.rp);
    load_planes<T>(sB1, b1p, K1, it.m + (int64_t)it.rt * t.r0 * it.m_ld, it.m_ld, it.m_ps, n1p, n1, it.rp);
    for (int q = 0; q < T; ++q) {  // Re_q -> slot 3q + 1, Im_q -> slot 3q + 2
        load_planes<1>(sB2 + (3 * q + 1) * b2p, b2p, K2, it.uth + q * it.uth_ps, it.uth_ld, it.uth_ps * T, sh.ntp,
                       nt, it.rt);
    }
    asm volatile("cp.async.commit_group;");
    asm volatile("cp.async.wait_group 0;");
    __syncthreads();
    for (int q = 0; q < T; ++q) {  // slot 3q = -Im_q (bfloat16 sign bits flipped)
        const uint4* src = reinterpret_cast<const uint4*>(sB2 + (3 * q + 2) * b2p);
        uint4* dst = reinterpret_cast<uint4*>(sB2 + 3 * q * b2p);
        for (int e = tid; e < b2p / 16; e += F34_THREADS) {
            const uint4 v = src[e];
            dst[e] = make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = tmem_base;
    // AG4 accumulator set b at d2 + b set: [re | im] of d0, then (two accumulators) of d1
    const uint32_t d2 = tm + 2 * sh.N1s;
    const int nbuf = sh.nbuf, set = 2 * sh.nacc * sh.ntp;
    bool ok = true;
    if (warp == F34_WORKERS / 32) {
        // ---- MMA warp: AG3 once, then AG4 for every r as soon as its A2 is written
        if (lane == 0) {
            issue_products<T>(tm, tm + sh.N1s, smem_u32(sA1), a1p, smem_u32(sB1), b1p, K1 * 16, K1 * 16, K1 / 16,
                              idesc_bf16(n1p));
            mma_commit(&mbar[F34_D1]);
            for (int j = 0; j < t.nr; ++j) {
                const int a = j & 1, b = j % nbuf;
                ok = mbar_wait(&mbar[F34_A2 + a], (j >> 1) & 1) && ok;
                if (j >= nbuf) ok = mbar_wait(&mbar[F34_EMPTY + b], ((j - nbuf) / nbuf) & 1) && ok;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dr = d2 + b * set;
                issue_products_cat<T>(dr, dr + (sh.nacc - 1) * 2 * sh.ntp, smem_u32(sA2b + a * 2 * T * a2p), a2p,
                                      smem_u32(sB2), b2p,
                                      K2 * 16, K2 * 16, K2 / 16, idesc_bf16(2 * sh.ntp));
                mma_commit(&mbar[F34_D2 + b]);
            }
        }
        __syncwarp();
    } else {
        // ---- workers: warps w, w + 4, ... share lane quarter w & 3 and split the columns
        const int phi = (warp & 3) * 32 + lane, grp = warp >> 2, ngrp = F34_WORKERS / 128;
        const bool rows = (warp & 3) * 32 < n_phi;  // quarters past n_phi hold no direction
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        const int64_t n_dir = c.n_dir;
        ok = mbar_wait(&mbar[F34_D1], 0);
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int j = 0; j <= t.nr; ++j) {
            if (j < t.nr) {
                // V_j: TMEM columns (a + r_t j) -> BF16 planes of A2[j & 1], row i_phi, depth a
                // (zeros past r_t); A2[j & 1] was last read by the MMAs of j - 2, waited below
                uint8_t* sA2 = sA2b + (j & 1) * 2 * T * a2p;
                if (rows)
                    for (int kc = grp; kc < K2 / 8; kc += ngrp) {
                        const int off = (phi >> 3) * (K2 * 16) + kc * 128 + (phi & 7) * 16;
                        if (kc * 8 >= it.rt) {
#pragma unroll
                            for (int q = 0; q < 2 * T; ++q)
                                *reinterpret_cast<uint4*>(sA2 + q * a2p + off) = make_uint4(0, 0, 0, 0);
                            continue;
                        }
                        uint32_t vr[8], vi[8], w[2 * T][4];
                        tmem_ld8(vr, tm + lanes + it.rt * j + kc * 8);
                        tmem_ld8(vi, tm + lanes + sh.N1s + it.rt * j + kc * 8);
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            uint32_t pr[3], pi[3];
                            const int k = kc * 8 + e;
                            split_pack<T>(k < it.rt ? __uint_as_float(vr[e]) : 0.f, k + 1 < it.rt ? __uint_as_float(vr[e + 1]) : 0.f, pr);
                            split_pack<T>(k < it.rt ? __uint_as_float(vi[e]) : 0.f, k + 1 < it.rt ? __uint_as_float(vi[e + 1]) : 0.f, pi);
#pragma unroll
                            for (int q = 0; q < T; ++q) {
                                w[q][e / 2] = pr[q];
                                w[T + q][e / 2] = pi[q];
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 2 * T; ++q)
                            *reinterpret_cast<uint4*>(sA2 + q * a2p + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
                    }
                asm volatile("fence.proxy.async.shared::cta;");
                mbar_arrive(&mbar[F34_A2 + (j & 1)]);
            }
            if (j > 0) {
                // spectra of RHS r0 + j - 1: TMEM -> rows in shared memory -> one contiguous block
                const int jj = j - 1, b = jj % nbuf;
                ok = mbar_wait(&mbar[F34_D2 + b], (jj / nbuf) & 1) && ok;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dr = d2 + b * set;
                for (int kc = grp; rows && kc < sh.ntp / 8; kc += ngrp) {
                    uint32_t vr[8], vi[8], ur[8] = {}, ui[8] = {};
                    tmem_ld8(vr, dr + lanes + kc * 8);
                    tmem_ld8(vi, dr + lanes + sh.ntp + kc * 8);
                    if (sh.nacc == 2) {
                        tmem_ld8(ur, dr + lanes + 2 * sh.ntp + kc * 8);
                        tmem_ld8(ui, dr + lanes + 3 * sh.ntp + kc * 8);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (phi < n_phi) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (kc * 8 + e < nt)
                                stage[phi * nt + kc * 8 + e] =
                                    make_float2(__uint_as_float(vr[e]) + __uint_as_float(ur[e]),
                                                __uint_as_float(vi[e]) + __uint_as_float(ui[e]));
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(&mbar[F34_EMPTY + b]);  // set b may take the MMAs of jj + nbuf
                workers_sync();
                float2* F = c.spec + (((int64_t)(t.r0 + jj) * c.G + it.g) * 2 + it.alpha) * n_dir;
                if ((n_dir & 1) == 0) {
                    const float4* src = reinterpret_cast<const float4*>(stage);
                    float4* dst = reinterpret_cast<float4*>(F);
                    for (int e = tid; e < (int)(n_dir >> 1); e += F34_WORKERS) dst[e] = src[e];
                } else {
                    for (int e = tid; e < (int)n_dir; e += F34_WORKERS) F[e] = stage[e];
                }
                workers_sync();
            }
        }
    }
    // every MMA was waited for (bounded) by the workers before TMEM is freed
    if (!ok) atomicAdd(c.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(sh.tcols));
}

// ------------------------------------------------- DG1a with (i_phi, r) as N
// P'_r[i_phi][a] = sum_theta conj(W g_r)[theta][i_phi] U_theta[theta][a] (Fig. 3b
// step 1, first factor) as D[a][(i_phi, r)]: U_theta^T is the A operand (the r_theta
// rows on the TMEM lanes), NP (i_phi, r) pairs of the weighted, conjugated FP32
// spectra are the B operand, split in registers.  One MMA then covers NP = 128 (or
// 64) pairs instead of r_theta columns.  The result goes TMEM -> shared memory ->
// the P'' planes [a + r_t r][i_phi] that DG1b reads.
struct D1Item {
    const bf16* uth; int64_t uth_ld, uth_ps;  // U_theta planes [a][i_theta]
    bf16* out; int64_t o_ld, o_ps;            // P'' planes [a + r_t r][i_phi]
    int g, alpha, rt;
};
struct D1Tile { int item, p0; };

constexpr int D1_THREADS = 256;

template <int T>
__global__ void __launch_bounds__(D1_THREADS) tc_dg1a_kernel(const TcCtx c, const D1Item* __restrict__ items,
                                                            const D1Tile* __restrict__ tiles, int K, int NP,
                                                            int AR, int tcols, int n_phi) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const D1Tile t = tiles[blockIdx.x];
    const D1Item it = items[t.item];
    const int nt = c.n_theta, npairs = n_phi * c.R;
    // A planes hold AR >= r_theta rows; the MMA reads 128 rows per plane, the rows past AR
    // (data of the next plane or of B, inside this CTA's shared memory) only reach lanes
    // past r_theta, which are never read back
    const int ap = AR * K * 2, bp = NP * K * 2;
    uint8_t* sA = smem;
    uint8_t* sB = smem + 2 * T * ap;
    float2* stage = reinterpret_cast<float2*>(sB);  // reused once the MMAs are done
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    // A: U_theta^T, r_theta rows (lanes past r_theta hold no output)
    load_planes<T>(sA, ap, K, it.uth, it.uth_ld, it.uth_ps, it.rt, it.rt, nt);
    asm volatile("cp.async.commit_group;");
    // B: pair row p0 + i = i_phi + n_phi r, depth theta; conj(W g), zero past n_theta and n_phi R.
    // Every load of a thread is issued before the splits (memory-level parallelism).
    const int kc8 = K / 8, ntask = NP * kc8;
    constexpr int ITER = 4;  // NP * K / 8 <= 4 * D1_THREADS (host check)
    float2 v[ITER][8];
#pragma unroll
    for (int u = 0; u < ITER; ++u) {
        const int task = tid + u * D1_THREADS, i = task / kc8, kc = task % kc8, p = t.p0 + i;
        const bool row_ok = task < ntask && p < npairs;
        const int ip = row_ok ? p % n_phi : 0, r = row_ok ? p / n_phi : 0;
        const int64_t o = (((int64_t)r * c.G + it.g) * 2 + it.alpha) * c.n_dir + (int64_t)nt * ip;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int th = kc * 8 + e;
            v[u][e] = make_float2(0.f, 0.f);
            if (row_ok && th < nt) {
                const float2 g = __ldg(c.spec_in + o + th);
                const float wt = c.w ? __ldg(c.w + th + (int64_t)nt * ip) : 1.0f;
                v[u][e] = make_float2(wt * g.x, -wt * g.y);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < ITER; ++u) {
        const int task = tid + u * D1_THREADS, i = task / kc8, kc = task % kc8;
        if (task >= ntask) break;
        uint32_t w[2 * T][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint32_t pr[3], pi[3];
            split_pack<T>(v[u][e].x, v[u][e + 1].x, pr);
            split_pack<T>(v[u][e].y, v[u][e + 1].y, pi);
#pragma unroll
            for (int q = 0; q < T; ++q) {
                w[q][e / 2] = pr[q];
                w[T + q][e / 2] = pi[q];
            }
        }
        const int off = (i >> 3) * (K * 16) + kc * 128 + (i & 7) * 16;
#pragma unroll
        for (int q = 0; q < 2 * T; ++q)
            *reinterpret_cast<uint4*>(sB + q * bp + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
    asm volatile("cp.async.wait_group 0;");
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = tmem_base;
    if (tid == 0) {
        issue_products<T>(tm, tm + NP, smem_u32(sA), ap, smem_u32(sB), bp, K * 16, K * 16, K / 16, idesc_bf16(NP));
        mma_commit(&mbar);
    }
    bool ok = mbar_wait(&mbar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(ok);
    if (ok) {
        // D[a][pair] -> stage[a][pair] (the warps whose lane quarter holds some a < r_theta)
        if (warp < 4 && warp * 32 < it.rt) {
            const uint32_t lanes = (uint32_t)(warp * 32) << 16;
            const int a = warp * 32 + lane;
            for (int c0 = 0; c0 < NP; c0 += 32) {
                uint32_t vr[32], vi[32];
                tmem_ld32(vr, tm + lanes + c0);
                tmem_ld32(vi, tm + lanes + NP + c0);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (a < it.rt) {
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        stage[a * NP + c0 + e] = make_float2(__uint_as_float(vr[e]), __uint_as_float(vi[e]));
                }
            }
        }
        __syncthreads();
        // stage -> P'' planes, row a + r_t r, column i_phi: eight pairs per task
        for (int task = tid; task < it.rt * (NP / 8); task += D1_THREADS) {
            const int a = task / (NP / 8), c8 = (task % (NP / 8)) * 8, p = t.p0 + c8;
            if (p >= npairs) continue;
            const int ip = p % n_phi, r = p / n_phi;
            const bool vec = ip + 8 <= n_phi && (ip & 7) == 0 && (it.o_ld & 7) == 0 && p + 8 <= npairs;
            if (vec) {
                uint32_t w[2 * T][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const float2 x0 = stage[a * NP + c8 + e], x1 = stage[a * NP + c8 + e + 1];
                    uint32_t pr[3], pi[3];
                    split_pack<T>(x0.x, x1.x, pr);
                    split_pack<T>(x0.y, x1.y, pi);
#pragma unroll
                    for (int q = 0; q < T; ++q) {
                        w[q][e / 2] = pr[q];
                        w[T + q][e / 2] = pi[q];
                    }
                }
                bf16* dst = it.out + (int64_t)(a + it.rt * r) * it.o_ld + ip;
#pragma unroll
                for (int q = 0; q < 2 * T; ++q)
                    *reinterpret_cast<uint4*>(dst + q * it.o_ps) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            } else {
                for (int e = 0; e < 8 && p + e < npairs; ++e) {
                    const int pe = p + e, ipe = pe % n_phi, re = pe / n_phi;
                    store_planes<T>(it.out, it.o_ps, (int64_t)(a + it.rt * re) * it.o_ld + ipe, stage[a * NP + c8 + e]);
                }
            }
        }
    } else {
        mbar_wait(&mbar, 0);  // no MMA may still run when TMEM is freed
        if (tid == 0) atomicAdd(c.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tcols));
}

// --------------------------------- narrow-N steps with the BF16 terms stacked along N
// DG1a  P'_r[i_phi][a] = sum_theta conj(W g_r)[theta][i_phi] U_theta[theta][a]   (Fig. 3b
//       step 1, first factor): rows m = i_phi + n_phi r on the TMEM lanes, A from the FP32
//       spectra (weighted, conjugated and split here), out the P'' planes [a + r_t r][i_phi];
// DG1b  H'_r[a][b] = sum_phi P'_r[i_phi][a] U_phi[i_phi][b]   (second factor): rows
//       m = a + r_t r, A the P'' planes, out the H planes [r][a + r_t b] that DG2 reads.
// N (r_theta or r_phi) is narrow, so the term products share MMAs: B stacks the BF16
// terms of the factor along N, Bpos = [Re_0 Im_0 Re_1 Im_1 ...] and Bneg = [-Im_0 Re_0
// -Im_1 Re_1 ...] (n8 = r8(rank) rows each), and term p of A multiplies the first T - p
// term pairs of B into the accumulator columns from 2 p n8 on,
//   A_p,re Bpos + A_p,im Bneg  ->  [L_p | ... | L_(T-1)],
// so that L_q (2 n8 columns, re | im) collects the products whose term orders add up
// to q: the leading hi x hi product alone in L_0, the corrections in their own
// accumulators, and the result is (L_2 + L_1) + L_0.  A K step of 16 takes 2T MMAs of
// N = 2 (T - p) n8 columns instead of 4 n_products narrow ones.  B is split here from
// the FP32 factor.  The epilogue writes the output planes straight from TMEM (one row
// per thread, consecutive rows on consecutive lanes).
struct CatItem {
    const float2* fac;               // U_theta (DG1a) or U_phi (DG1b): K x rank, column-major (FP32)
    const bf16* a; int64_t a_ld, a_ps;  // DG1b: P'' planes [a + r_t r][i_phi]
    bf16* out; int64_t o_ld, o_ps;   // P'' (DG1a) or H (DG1b) planes
    int g, alpha, rt, rank, M;       // rank = N of this item; M = rows (n_phi R or r_t R)
};

constexpr int CAT_THREADS = 256;
constexpr int CAT_ITER = 4;  // DG1a A loads per thread: 128 rows x K16 / 8 <= 4 x CAT_THREADS (host check)
enum { CAT_DG1A = 0, CAT_DG1B = 1 };

// byte offset of 16-byte chunk kc of row `row` in the canonical no-swizzle K-major layout
__device__ __forceinline__ int canon_off(int row, int kc, uint32_t sbo) {
    return (row >> 3) * (int)sbo + kc * 128 + (row & 7) * 16;
}

// DG1a A, rows p0 .. p0 + 127 = (i_phi, r) pairs, depth theta: conj(W g) loaded into
// registers (zero past n_theta and the item's rows)
__device__ __forceinline__ void cat_load_g(float2 (&v)[CAT_ITER][8], const TcCtx& c, const CatItem& it, int p0,
                                           int kc8, int n_phi) {
    const int nt = c.n_theta, ntask = TBM * kc8;
#pragma unroll
    for (int u = 0; u < CAT_ITER; ++u) {
        const int task = threadIdx.x + u * CAT_THREADS, i = task / kc8, kc = task % kc8, p = p0 + i;
        const bool row_ok = task < ntask && p < it.M;
        const int ip = row_ok ? p % n_phi : 0, r = row_ok ? p / n_phi : 0;
        const int64_t o = (((int64_t)r * c.G + it.g) * 2 + it.alpha) * c.n_dir + (int64_t)nt * ip;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int th = kc * 8 + e;
            v[u][e] = make_float2(0.f, 0.f);
            if (row_ok && th < nt) {
                const float2 g = __ldg(c.spec_in + o + th);
                const float wt = c.w ? __ldg(c.w + th + (int64_t)nt * ip) : 1.0f;
                v[u][e] = make_float2(wt * g.x, -wt * g.y);
            }
        }
    }
}

// the loaded DG1a A values, split into 2T planes of the canonical layout
template <int T>
__device__ __forceinline__ void cat_store_g(uint8_t* sA, const float2 (&v)[CAT_ITER][8], int kc8, uint32_t sbo,
                                            int planeA) {
    const int ntask = TBM * kc8;
#pragma unroll
    for (int u = 0; u < CAT_ITER; ++u) {
        const int task = threadIdx.x + u * CAT_THREADS, i = task / kc8, kc = task % kc8;
        if (task >= ntask) break;
        uint32_t w[2 * T][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint32_t pr[3], pi[3];
            split_pack<T>(v[u][e].x, v[u][e + 1].x, pr);
            split_pack<T>(v[u][e].y, v[u][e + 1].y, pi);
#pragma unroll
            for (int q = 0; q < T; ++q) {
                w[q][e / 2] = pr[q];
                w[T + q][e / 2] = pi[q];
            }
        }
        const int off = canon_off(i, kc, sbo);
#pragma unroll
        for (int q = 0; q < 2 * T; ++q)
            *reinterpret_cast<uint4*>(sA + q * planeA + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

// DG1b A: rows p0 .. p0 + 127 of the P'' planes, 16-byte chunks by cp.async (zero past the
// item's rows and past the planes' leading dimension, whose padding columns are zero)
template <int T>
__device__ __forceinline__ void cat_load_planes(uint8_t* sA, const CatItem& it, int p0, int kc8, uint32_t sbo,
                                                int planeA) {
    const int ntask = TBM * kc8;
    for (int task = threadIdx.x; task < 2 * T * ntask; task += CAT_THREADS) {
        const int q = task / ntask, rem = task % ntask, i = rem / kc8, kc = rem % kc8, m = p0 + i;
        uint8_t* dst = sA + q * planeA + canon_off(i, kc, sbo);
        const bool ok = m < it.M && kc * 8 < it.a_ld;
        const bf16* src = ok ? it.a + q * it.a_ps + (int64_t)m * it.a_ld + kc * 8 : it.a;
        cp16(dst, src, ok ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;");
}

// B: row n of slot j, depth k, from the factor (zero past its rank and K)
template <int T>
__device__ __forceinline__ void cat_build_b(uint8_t* sBp, uint8_t* sBn, const CatItem& it, int K, int kc8,
                                            uint32_t sbo) {
    const int n8 = (it.rank + 7) & ~7;
    for (int task = threadIdx.x; task < n8 * kc8; task += CAT_THREADS) {
        const int n = task / kc8, kc = task % kc8;
        uint32_t wr[T][4], wi[T][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float2 u0 = make_float2(0.f, 0.f), u1 = u0;
            const int k = kc * 8 + e;
            if (n < it.rank && k < K) u0 = __ldg(it.fac + k + (int64_t)K * n);
            if (n < it.rank && k + 1 < K) u1 = __ldg(it.fac + k + 1 + (int64_t)K * n);
            uint32_t pr[3], pi[3];
            split_pack<T>(u0.x, u1.x, pr);
            split_pack<T>(u0.y, u1.y, pi);
#pragma unroll
            for (int q = 0; q < T; ++q) {
                wr[q][e / 2] = pr[q];
                wi[q][e / 2] = pi[q];
            }
        }
#pragma unroll
        for (int q = 0; q < T; ++q) {
            const uint4 re = make_uint4(wr[q][0], wr[q][1], wr[q][2], wr[q][3]);
            const uint4 im = make_uint4(wi[q][0], wi[q][1], wi[q][2], wi[q][3]);
            // the split is odd in its argument: the terms of -Im are the terms of Im, negated
            const uint4 nim = make_uint4(im.x ^ 0x80008000u, im.y ^ 0x80008000u, im.z ^ 0x80008000u,
                                         im.w ^ 0x80008000u);
            *reinterpret_cast<uint4*>(sBp + canon_off((2 * q) * n8 + n, kc, sbo)) = re;
            *reinterpret_cast<uint4*>(sBp + canon_off((2 * q + 1) * n8 + n, kc, sbo)) = im;
            *reinterpret_cast<uint4*>(sBn + canon_off((2 * q) * n8 + n, kc, sbo)) = nim;
            *reinterpret_cast<uint4*>(sBn + canon_off((2 * q + 1) * n8 + n, kc, sbo)) = re;
        }
    }
}

// the 2T MMAs per K step of the stacked product into the accumulator at TMEM column d0
// (one thread)
template <int T>
__device__ __forceinline__ void cat_issue(uint32_t d0, const uint8_t* sA, const uint8_t* sBp, const uint8_t* sBn,
                                          int n8, int K16, uint32_t sbo, int planeA) {
    const uint64_t da = make_desc_sbo(smem_u32(sA), sbo), dbp = make_desc_sbo(smem_u32(sBp), sbo),
                   dbn = make_desc_sbo(smem_u32(sBn), sbo);
    for (int ks = 0; ks < K16 / 16; ++ks)
#pragma unroll
        for (int p = 0; p < T; ++p) {
            const uint32_t idesc = idesc_bf16(2 * (T - p) * n8);
            const uint64_t ar = da + (uint32_t)(p * planeA + ks * 256) / 16;
            const uint64_t ai = da + (uint32_t)((T + p) * planeA + ks * 256) / 16;
            const uint32_t d = d0 + (uint32_t)(2 * p * n8);
            mma_bf16(d, ar, dbp + (uint32_t)(ks * 256) / 16, idesc, (ks > 0 || p > 0) ? 1u : 0u);
            mma_bf16(d, ai, dbn + (uint32_t)(ks * 256) / 16, idesc, 1u);
        }
}

// (L_2 + L_1) + L_0 of the accumulator at TMEM column d0 -> the output planes: warps w
// and w + 4 read lane quarter w & 3, alternate blocks of 8 columns each.  Output element
// (m, column n): DG1a row n + r_t r, column i_phi of P''; DG1b row r, column a + r_t n of H.
template <int T, int MODE>
__device__ __forceinline__ void cat_epilogue(uint32_t d0, const CatItem& it, int p0, int n_phi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n8 = (it.rank + 7) & ~7;
    const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
    const int m = p0 + (warp & 3) * 32 + lane;
    const bool row_ok = m < it.M;
    int64_t base = 0, step = 0;
    if (row_ok) {
        if (MODE == CAT_DG1A) {
            base = (int64_t)it.rt * (m / n_phi) * it.o_ld + m % n_phi;
            step = it.o_ld;
        } else {
            base = (int64_t)(m / it.rt) * it.o_ld + m % it.rt;
            step = it.rt;
        }
    }
    for (int c0 = (warp >> 2) * 8; c0 < n8; c0 += 16) {
        uint32_t vr[T][8], vi[T][8];
#pragma unroll
        for (int q = 0; q < T; ++q) {
            tmem_ld8(vr[q], d0 + lanes + (uint32_t)(2 * q * n8 + c0));
            tmem_ld8(vi[q], d0 + lanes + (uint32_t)(2 * q * n8 + n8 + c0));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (!row_ok) continue;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int n = c0 + e;
            if (n >= it.rank) break;
            float re = __uint_as_float(vr[T - 1][e]), im = __uint_as_float(vi[T - 1][e]);
#pragma unroll
            for (int q = T - 2; q >= 0; --q) {
                re += __uint_as_float(vr[q][e]);
                im += __uint_as_float(vi[q][e]);
            }
            store_planes<T>(it.out, it.o_ps, base + step * n, make_float2(re, im));
        }
    }
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int tcols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

// One 128-row tile per CTA.
template <int T, int MODE>
__global__ void __launch_bounds__(CAT_THREADS) tc_cat_kernel(const TcCtx c, const CatItem* __restrict__ items,
                                                            const D1Tile* __restrict__ tiles, int K, int K16,
                                                            int n8max, int tcols, int n_phi) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const D1Tile t = tiles[blockIdx.x];
    const CatItem it = items[t.item];
    const int kc8 = K16 / 8;
    const uint32_t sbo = (uint32_t)K16 * 16;            // bytes from one 8-row group to the next
    const int planeA = TBM / 8 * (int)sbo;              // one term plane of A (128 rows)
    const int bbuf = 2 * T * n8max / 8 * (int)sbo;      // Bpos or Bneg
    uint8_t* sA = smem;
    uint8_t* sBp = smem + 2 * T * planeA;
    uint8_t* sBn = sBp + bbuf;
    if (warp == 0) tmem_alloc(&tmem_base, tcols);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    // A's loads first, B built while they are in flight
    if constexpr (MODE == CAT_DG1A) {
        float2 v[CAT_ITER][8];
        cat_load_g(v, c, it, t.p0, kc8, n_phi);
        cat_build_b<T>(sBp, sBn, it, K, kc8, sbo);
        cat_store_g<T>(sA, v, kc8, sbo, planeA);
    } else {
        cat_load_planes<T>(sA, it, t.p0, kc8, sbo, planeA);
        cat_build_b<T>(sBp, sBn, it, K, kc8, sbo);
        asm volatile("cp.async.wait_group 0;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = tmem_base;
    if (tid == 0) {
        cat_issue<T>(tm, sA, sBp, sBn, (it.rank + 7) & ~7, K16, sbo, planeA);
        mma_commit(&mbar);
    }
    bool ok = mbar_wait(&mbar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(ok);
    if (ok) {
        cat_epilogue<T, MODE>(tm, it, t.p0, n_phi);
    } else {
        mbar_wait(&mbar, 0);  // no MMA may still run when TMEM is freed
        if (tid == 0) atomicAdd(c.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tcols));
}

// ------------------------------------------------------------ operand prep
// Split planes of an FP32 complex matrix: dst[p][r][k] for r < rows, k < cols,
// src element (r, k) at src[r * sr + k * sk]; entries k in [cols, ld) stay as they are.
// inner > 0: row r of the planes is source row (r / inner) + outer (r % inner) (the rows
// of C_(3)^T, index a + r_t b, taken in the order b + r_p a).
template <int T>
__global__ void planes_kernel(const float2* __restrict__ src, int rows, int cols, int64_t sr, int64_t sk,
                              bf16* __restrict__ dst, int64_t ld, int64_t ps, int inner, int outer) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), k = (int)(e % cols);
        const int rs = inner > 0 ? r / inner + outer * (r % inner) : r;
        store_planes<T>(dst, ps, (int64_t)r * ld + k, src[(int64_t)rs * sr + (int64_t)k * sk]);
    }
}

// X_g planes [r][n] for every group: x[grp_rwg[off_g + n] + ldx r].
template <int T>
__global__ void prep_x_kernel(const float2* __restrict__ x, int64_t ldx, const int* __restrict__ grp_rwg,
                              const TcProb* __restrict__ probs, int n_probs, int R) {
    for (int q = blockIdx.y; q < n_probs; q += gridDim.y) {
        const TcProb& p = probs[q];  // AG1 problem of (g, alpha = 0): B0 points at the group's X planes
        if (p.alpha != 0) continue;
        bf16* dst = const_cast<bf16*>(p.B0);
        const int nb = p.K0;
        const int64_t total = (int64_t)R * nb;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
            const int r = (int)(e / nb), n = (int)(e % nb);
            store_planes<T>(dst, p.b_ps0, (int64_t)r * p.b_ld0 + n, x[(int64_t)grp_rwg[p.rwg + n] + ldx * r]);
        }
    }
}

// G' planes [i_phi + n_phi r][i_theta] = conj(W g) for every (g, alpha).
template <int T>
__global__ void prep_g_kernel(const float2* __restrict__ spec, const float* __restrict__ w,
                              const TcProb* __restrict__ probs, int n_probs, int R, int G, int n_theta, int n_phi) {
    const int n_dir = n_theta * n_phi;
    for (int q = blockIdx.y; q < n_probs; q += gridDim.y) {
        const TcProb& p = probs[q];  // DG1a problem: A0 points at the item's G' planes
        bf16* dst = const_cast<bf16*>(p.A0);
        const int64_t total = (int64_t)R * n_dir;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
            const int r = (int)(e / n_dir), o = (int)(e % n_dir);
            const int it = o % n_theta, ip = o / n_theta;
            const float2 v = spec[(((int64_t)r * G + p.g) * 2 + p.alpha) * n_dir + o];
            const float wt = w ? w[o] : 1.0f;
            store_planes<T>(dst, p.a_ps0, (int64_t)(ip + n_phi * r) * p.a_ld0 + it, make_float2(wt * v.x, -wt * v.y));
        }
    }
}

int g1d(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096)); }

int64_t r8(int64_t v) { return (v + 7) & ~int64_t(7); }

// Leading and correction products in separate TMEM accumulators (TFMM_TC_HSPLIT=0 turns it off).
bool tc_split_accumulators() {
    static const bool on = [] {
        const char* e = std::getenv("TFMM_TC_HSPLIT");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Raises a kernel's dynamic shared-memory limit, once per (device, kernel): the
// attribute belongs to the current device's context.
void allow_dyn_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int dev = 0;
    TFMM_CUDA_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, kernel})) return;
    TFMM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.insert({dev, kernel});
}

// k-tiles (of 32) per chunk of the chunked accumulation (TFMM_TC_CHUNK, default 2,
// i.e. 4 K steps of 16 per accumulator; 0 turns chunking off).
int tc_chunk_ktiles() {
    static const int v = [] {
        const char* e = std::getenv("TFMM_TC_CHUNK");
        return e ? std::max(0, std::atoi(e)) : 2;
    }();
    return v;
}

// Ring depth and TMEM columns from the stage's largest K and BN; shared memory is
// padded so that the CTAs one SM can hold never ask for more than its 512 columns.
// Stages whose K is longer than one chunk (AG1, AG2, DG1b, DG2, DG3) run the chunked
// accumulation.
template <int T, int S>
void launch_tc(const TcStagePlan& st, const TcCtx& c, cudaStream_t s) {
    if (st.n_tiles == 0) return;
    constexpr int NST_MAX = (T == 2) ? 3 : 2;
    constexpr size_t STAGE = (size_t)2 * 2 * T * PLANE_TILE;
    const int nst = std::max(1, std::min(NST_MAX, st.max_kt));
    const int cofs = (st.max_bn + 31) / 32 * 32;
    const int hsplit = tc_split_accumulators() ? 1 : 0;
    int tcols = 32;
    while (tcols < (hsplit ? 4 : 2) * cofs) tcols *= 2;
    // at most 512 / tcols CTAs per SM: pad the shared memory request so that no more fit
    const int ctas_tmem = 512 / tcols;
    constexpr size_t kSmemSM = 228 * 1024, kMaxDyn = 225 * 1024;
    size_t smem = nst * STAGE;
    if (kSmemSM / (smem + 2048) > (size_t)ctas_tmem) smem = std::min(kMaxDyn, kSmemSM / ctas_tmem - 2048);
    const int chunk = tc_chunk_ktiles();
    const TcProb* probs = reinterpret_cast<const TcProb*>(st.d_probs);
    if (st.d_maps && hsplit) {
        // TMA-fed ring of K steps of 16: as many stages as fit next to nothing else
        const size_t stage = (size_t)2 * 8 * 2 * T * 2 * (TBM + st.max_bn);
        const int nst_tma = (int)std::min<size_t>(NST_TMA_MAX, kMaxDyn / stage);
        allow_dyn_smem(reinterpret_cast<const void*>(tc_gemm_tma_kernel<T, S>), kMaxDyn);
        tc_gemm_tma_kernel<T, S><<<st.n_tiles, 2 * TTHREADS, nst_tma * stage, s>>>(
            c, probs, static_cast<const CUtensorMap*>(st.d_maps), st.d_tiles, nst_tma, tcols, cofs,
            chunk > 0 ? chunk : 1 << 30);
        TFMM_CUDA_CHECK(cudaGetLastError());
        return;
    }
    if constexpr (S == TAG1 || S == TAG2 || S == TDG1B || S == TDG2 || S == TDG3) {
        if (hsplit && chunk > 0 && st.max_kt > chunk) {
            allow_dyn_smem(reinterpret_cast<const void*>(tc_gemm_kernel<T, S, true>), kMaxDyn);
            tc_gemm_kernel<T, S, true><<<st.n_tiles, 2 * TTHREADS, smem, s>>>(c, probs, st.d_tiles, nst, tcols, cofs,
                                                                             hsplit, chunk);
            TFMM_CUDA_CHECK(cudaGetLastError());
            return;
        }
    }
    allow_dyn_smem(reinterpret_cast<const void*>(tc_gemm_kernel<T, S, false>), kMaxDyn);
    tc_gemm_kernel<T, S, false><<<st.n_tiles, TTHREADS, smem, s>>>(c, probs, st.d_tiles, nst, tcols, cofs, hsplit, 1);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

}  // namespace

TcStagePlan::~TcStagePlan() {
    if (d_probs) cudaFree(d_probs);
    if (d_tiles) cudaFree(d_tiles);
    if (d_maps) cudaFree(d_maps);
}

TcPlan::~TcPlan() {
    for (auto* b : buf)
        if (b) cudaFree(b);
}

// BF16 planes of every factor in the two K-major layouts the chains read.
void build_tc_factors(Plan& P, int T, cudaStream_t s) {
    if (P.tc_fac[T].p) return;
    std::vector<TcItem>& items = P.tc_items[T];
    const int nt = P.n_theta, np = P.n_phi;
    items.assign(P.items.size(), TcItem{});
    int64_t off = 0;
    auto add = [&](TcMat& m, int rows, int cols) {
        m.rows = rows;
        m.ld = r8(cols);
        m.off = off;
        off += (int64_t)2 * T * rows * m.ld;
        off = (off + 63) & ~int64_t(63);
    };
    for (size_t q = 0; q < P.items.size(); ++q) {
        const TuckerItem& d = P.items[q];
        TcItem& t = items[q];
        const int m = d.rt * d.rp;
        add(t.ubT, d.rb, d.n_beta);   // [c][n]
        add(t.ub, d.n_beta, d.rb);    // [n][c]
        add(t.c3T, m, d.rb);          // [ab][c], rows in the order b + r_p a
        add(t.c3, d.rb, m);           // [c][ab]
        add(t.uphT, np, d.rp);        // [i_phi][b]
        add(t.uph, d.rp, np);         // [b][i_phi]
        add(t.uthT, nt, d.rt);        // [i_theta][a]
        add(t.uth, d.rt, nt);         // [a][i_theta]
    }
    TFMM_CUDA_CHECK(device_malloc(&P.tc_fac[T].p, sizeof(bf16) * std::max<int64_t>(off, 1)));
    TFMM_CUDA_CHECK(cudaMemsetAsync(P.tc_fac[T].p, 0, sizeof(bf16) * std::max<int64_t>(off, 1), s));
    bf16* base = reinterpret_cast<bf16*>(P.tc_fac[T].p);
    auto conv = [&](const float2* src, int rows, int cols, int64_t sr, int64_t sk, const TcMat& m, int inner = 0,
                    int outer = 0) {
        const int64_t ps = (int64_t)m.rows * m.ld;
        if (T == 2)
            planes_kernel<2><<<g1d((int64_t)rows * cols), 256, 0, s>>>(src, rows, cols, sr, sk, base + m.off, m.ld, ps,
                                                                       inner, outer);
        else
            planes_kernel<3><<<g1d((int64_t)rows * cols), 256, 0, s>>>(src, rows, cols, sr, sk, base + m.off, m.ld, ps,
                                                                       inner, outer);
    };
    for (size_t q = 0; q < P.items.size(); ++q) {
        const TuckerItem& d = P.items[q];
        const TcItem& t = items[q];
        const int m = d.rt * d.rp;
        const float2* ub = P.d_factors + d.ub;      // U_beta^T rows: (c, n) at c ld_nb + n
        const float2* cc = P.d_factors + d.core;    // C_(3) rows:    (c, ab) at c ld_ab + ab
        const float2* up = P.d_factors + d.uphi;    // U_phi:         (i_phi, b) at i_phi + n_phi b
        const float2* ut = P.d_factors + d.uth;     // U_theta:       (i_theta, a) at i_theta + n_theta a
        conv(ub, d.rb, d.n_beta, d.ld_nb, 1, t.ubT);
        conv(ub, d.n_beta, d.rb, 1, d.ld_nb, t.ub);
        conv(cc, m, d.rb, 1, d.ld_ab, t.c3T, d.rp, d.rt);  // rows b + r_p a: AG2 writes M' in runs of b
        conv(cc, d.rb, m, d.ld_ab, 1, t.c3);
        conv(up, np, d.rp, 1, np, t.uphT);
        conv(up, d.rp, np, np, 1, t.uph);
        conv(ut, nt, d.rt, 1, nt, t.uthT);
        conv(ut, d.rt, nt, nt, 1, t.uth);
    }
    TFMM_CUDA_CHECK(cudaGetLastError());
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
    if (!P.tc_err.p) {
        TFMM_CUDA_CHECK(device_malloc(&P.tc_err.p, sizeof(int)));
        TFMM_CUDA_CHECK(cudaMemset(P.tc_err.p, 0, sizeof(int)));
    }
}

namespace {

void add_tc_tiles(std::vector<MrTile>& tiles, int prob, int M, int N) {
    for (int m0 = 0; m0 < M; m0 += TBM)
        for (int n0 = 0; n0 < N; n0 += TBN_MAX) tiles.push_back(MrTile{prob, m0, n0});
}

int bn_of(int N) { return (int)std::min<int64_t>(TBN_MAX, (N + 15) / 16 * 16); }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// 3-D map of the 2T planes of a K-major matrix (K x rows x planes, boxes of 8 K x
// box_rows x 2T); false when the layout breaks a rule of the copy engine.
bool encode_planes(CUtensorMap* m, const bf16* base, int64_t K, int64_t rows, int64_t ld, int64_t ps, int T,
                   int box_rows) {
    const auto fn = tensor_map_encoder();
    if (!fn || !base || K < 1 || rows < 1 || ld < K || ld % 8 || ps % 8 || ps < rows * ld ||
        reinterpret_cast<uintptr_t>(base) % 16)
        return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)(2 * T)};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ps * 2};
    cuuint32_t box[3] = {8, (cuuint32_t)box_rows, (cuuint32_t)(2 * T)};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps (A0, B0, A1, B1) of every problem of a stage for tc_gemm_tma_kernel; the
// stage keeps the cp.async kernel when one cannot be made or TFMM_TC_TMA=0.
void build_stage_maps(TcStagePlan& st, const std::vector<TcProb>& probs, int T) {
    if (const char* e = std::getenv("TFMM_TC_TMA"); e && e[0] == '0') return;
    if (probs.empty()) return;
    std::vector<CUtensorMap> maps(4 * probs.size());
    for (size_t i = 0; i < probs.size(); ++i) {
        const TcProb& p = probs[i];
        CUtensorMap* m = &maps[4 * i];
        bool ok = encode_planes(m + 0, p.A0, p.K0, p.M, p.a_ld0, p.a_ps0, T, TBM) &&
                  encode_planes(m + 1, p.B0, p.K0, p.N, p.b_ld0, p.b_ps0, T, p.BN);
        if (ok && p.K1 > 0)
            ok = encode_planes(m + 2, p.A1, p.K1, p.M, p.a_ld1, p.a_ps1, T, TBM) &&
                 encode_planes(m + 3, p.B1, p.K1, p.N, p.b_ld1, p.b_ps1, T, p.BN);
        else {
            m[2] = m[0];
            m[3] = m[1];
        }
        if (!ok) return;
    }
    TFMM_CUDA_CHECK(device_malloc(&st.d_maps, sizeof(CUtensorMap) * maps.size()));
    TFMM_CUDA_CHECK(cudaMemcpy(st.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
}

void upload_tc_stage(TcStagePlan& st, const std::vector<TcProb>& probs, const std::vector<MrTile>& tiles) {
    st.n_tiles = (int)tiles.size();
    st.n_probs = (int)probs.size();
    st.max_kt = 1;
    st.max_bn = 16;
    for (const auto& p : probs) {
        const int kt = (p.K0 + TBK - 1) / TBK + (p.K1 > 0 ? (p.K1 + TBK - 1) / TBK : 0);
        st.max_kt = std::max(st.max_kt, kt);
        st.max_bn = std::max(st.max_bn, p.BN);
    }
    TFMM_CUDA_CHECK(device_malloc(&st.d_probs, sizeof(TcProb) * std::max<size_t>(probs.size(), 1)));
    TFMM_CUDA_CHECK(device_malloc(&st.d_tiles, sizeof(MrTile) * std::max<size_t>(tiles.size(), 1)));
    TFMM_CUDA_CHECK(cudaMemcpy(st.d_probs, probs.data(), sizeof(TcProb) * probs.size(), cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(cudaMemcpy(st.d_tiles, tiles.data(), sizeof(MrTile) * tiles.size(), cudaMemcpyHostToDevice));
}

bool fused_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("TFMM_TC_FUSED");
        return !(e && e[0] == '0');
    }();
    return on;
}

constexpr size_t kMaxDynSmem = 225 * 1024;

size_t f34_smem(int T, int K1, int K2, int N1p, int ntp, int nt, int np) {
    const size_t pl = (size_t)2 * T * 2;  // bytes per element over the 2T planes
    return std::max(pl * TBM * K1, (size_t)np * nt * 8) + pl * std::max((size_t)N1p * K1, (size_t)2 * TBM * K2) +
           (size_t)3 * T * 2 * ntp * K2;
}

// Shapes and work list of the fused AG3 + AG4 kernel; leaves M.fused34 false
// when some item cannot run in one CTA (n_phi > 128 lanes, TMEM or shared memory).
template <class MOff>
void plan_fused34(const Plan& P, TcPlan& M, const bf16* F, const std::vector<TcItem>& tci, const bf16* Mb, MOff moff) {
    M.fused34 = false;
    if (!fused_enabled()) return;
    const int T = M.T, R = M.R, nt = P.n_theta, np = P.n_phi;
    if (np > TBM || nt > 128) return;  // lanes; AG4 runs as one MMA of N = 2 n_theta (<= 256)
    FusedShape f;
    f.K1 = (P.max_rank[1] + 15) & ~15;
    f.K2 = (P.max_rank[0] + 15) & ~15;
    f.ntp = (nt + 15) & ~15;
    f.nt32 = (nt + 31) & ~31;
    // two AG4 accumulator sets in flight (the MMAs of r overlap the spectra of r - 1), one
    // accumulator each; both are tuning knobs
    f.nbuf = 2;
    f.nacc = 1;
    if (const char* e = std::getenv("TFMM_TC_F34_NBUF")) f.nbuf = (std::atoi(e) == 1) ? 1 : 2;
    if (const char* e = std::getenv("TFMM_TC_F34_NACC")) f.nacc = (std::atoi(e) == 2) ? 2 : 1;
    const int n1s_cap = ((512 - f.nbuf * 2 * f.nacc * f.ntp) / 2) & ~31;
    int n1max = std::min(256, n1s_cap);
    if (const char* e = std::getenv("TFMM_TC_F34_N1")) n1max = std::min(n1max, std::max(16, std::atoi(e)) & ~15);
    if (P.tc_f34_n1 > 0) n1max = std::min(n1max, std::max(16, P.tc_f34_n1) & ~15);
    while (n1max >= 16 && f34_smem(T, f.K1, f.K2, n1max, f.ntp, nt, np) > kMaxDynSmem) n1max -= 16;
    if (n1max < ((P.max_rank[0] + 15) & ~15)) return;
    std::vector<F34Item> items(P.items.size());
    std::vector<int> nr_of(P.items.size());
    int n1p_max = 16;
    for (size_t q = 0; q < P.items.size(); ++q) {
        const TuckerItem& d = P.items[q];
        const TcItem& ti = tci[q];
        F34Item& it = items[q];
        it.uph = F + ti.uphT.off; it.uph_ld = ti.uphT.ld; it.uph_ps = (int64_t)ti.uphT.rows * ti.uphT.ld;
        it.uth = F + ti.uthT.off; it.uth_ld = ti.uthT.ld; it.uth_ps = (int64_t)ti.uthT.rows * ti.uthT.ld;
        it.m = Mb + moff((int)q); it.m_ld = r8(d.rp); it.m_ps = (int64_t)d.rt * R * r8(d.rp);
        it.g = d.g; it.alpha = d.alpha; it.rt = d.rt; it.rp = d.rp;
        const int nr = std::max(1, std::min(R, n1max / d.rt));
        nr_of[q] = nr;
        n1p_max = std::max(n1p_max, (d.rt * nr + 15) & ~15);
    }
    f.N1p = n1p_max;
    f.N1s = (n1p_max + 31) & ~31;
    f.tcols = 32;
    while (f.tcols < 2 * f.N1s + f.nbuf * 2 * f.nacc * f.ntp) f.tcols *= 2;
    if (f.tcols > 512) return;
    f.smem = f34_smem(T, f.K1, f.K2, f.N1p, f.ntp, nt, np);
    // no more CTAs per SM than their TMEM allocations allow
    constexpr size_t kSmemSM = 228 * 1024;
    const int ctas_tmem = 512 / f.tcols;
    if (kSmemSM / (f.smem + 2048) > (size_t)ctas_tmem) f.smem = std::min(kMaxDynSmem, kSmemSM / ctas_tmem - 2048);
    // work list, most work first
    std::vector<int> order(P.items.size());
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int q) { return (double)P.items[q].rt * (P.items[q].rp + nt); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<F34Tile> tiles;
    for (int q : order)
        for (int r0 = 0; r0 < R; r0 += nr_of[q]) tiles.push_back(F34Tile{q, r0, std::min(nr_of[q], R - r0)});
    TFMM_CUDA_CHECK(device_malloc(&M.f34_items.p, sizeof(F34Item) * items.size()));
    TFMM_CUDA_CHECK(device_malloc(&M.f34_tiles.p, sizeof(F34Tile) * tiles.size()));
    TFMM_CUDA_CHECK(cudaMemcpy(M.f34_items.p, items.data(), sizeof(F34Item) * items.size(), cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(cudaMemcpy(M.f34_tiles.p, tiles.data(), sizeof(F34Tile) * tiles.size(), cudaMemcpyHostToDevice));
    M.f34_ntiles = (int)tiles.size();
    M.f34 = f;
    M.fused34 = true;
}

template <int T>
void launch_ag34(const Plan& P, const TcPlan& M, const TcCtx& c, cudaStream_t s) {
    allow_dyn_smem(reinterpret_cast<const void*>(tc_ag34_kernel<T>), kMaxDynSmem);
    tc_ag34_kernel<T><<<M.f34_ntiles, F34_THREADS, M.f34.smem, s>>>(
        c, static_cast<const F34Item*>(M.f34_items.p), static_cast<const F34Tile*>(M.f34_tiles.p), M.f34, P.n_phi);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

// DG1a with the (i_phi, r) pairs as N: NP = 128 pairs per CTA when shared memory allows,
// else 64; leaves M.dg1a false when neither fits (the generic stage kernel runs instead).
template <class VOff>
void plan_dg1a(const Plan& P, TcPlan& M, const bf16* F, const std::vector<TcItem>& tci, bf16* Vb, VOff voff) {
    M.dg1a = false;
    if (!fused_enabled()) return;
    if (const char* e = std::getenv("TFMM_TC_DG1A"); e && e[0] == '0') return;
    const int T = M.T, R = M.R, nt = P.n_theta, np = P.n_phi;
    if (P.max_rank[0] > TBM) return;
    const int K = (nt + 15) & ~15;
    const int AR = (int)r8(P.max_rank[0]);
    // 128 pairs per CTA (two CTAs per SM when shared memory allows), else 64; the staged
    // result (r_theta x NP complex) reuses B, the loads are at most 4 tasks per thread
    int NP = 0;
    for (int cand : {128, 64}) {
        if (P.tc_dg1a_pairs > 0 && cand != P.tc_dg1a_pairs) continue;
        const size_t smem = (size_t)2 * T * 2 * K * (AR + cand);
        const bool stage_fits = (size_t)P.max_rank[0] * cand * 8 <= (size_t)2 * T * 2 * K * cand;
        const bool overread_fits = (size_t)2 * T * cand >= TBM;  // B covers the A planes' rows past AR
        const bool tasks_fit = cand * (K / 8) <= 4 * D1_THREADS;
        if (smem <= kMaxDynSmem && stage_fits && overread_fits && tasks_fit) {
            NP = cand;
            break;
        }
    }
    if (NP == 0) return;
    std::vector<D1Item> items(P.items.size());
    for (size_t q = 0; q < P.items.size(); ++q) {
        const TuckerItem& d = P.items[q];
        const TcMat& u = tci[q].uth;
        D1Item& it = items[q];
        it.uth = F + u.off; it.uth_ld = u.ld; it.uth_ps = (int64_t)u.rows * u.ld;
        it.out = Vb + voff((int)q); it.o_ld = r8(np); it.o_ps = (int64_t)d.rt * R * r8(np);
        it.g = d.g; it.alpha = d.alpha; it.rt = d.rt;
    }
    std::vector<D1Tile> tiles;
    const int npairs = np * R;
    for (size_t q = 0; q < P.items.size(); ++q)
        for (int p0 = 0; p0 < npairs; p0 += NP) tiles.push_back(D1Tile{(int)q, p0});
    TFMM_CUDA_CHECK(device_malloc(&M.dg1a_items.p, sizeof(D1Item) * items.size()));
    TFMM_CUDA_CHECK(device_malloc(&M.dg1a_tiles.p, sizeof(D1Tile) * tiles.size()));
    TFMM_CUDA_CHECK(cudaMemcpy(M.dg1a_items.p, items.data(), sizeof(D1Item) * items.size(), cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(cudaMemcpy(M.dg1a_tiles.p, tiles.data(), sizeof(D1Tile) * tiles.size(), cudaMemcpyHostToDevice));
    M.dg1a_ntiles = (int)tiles.size();
    M.dg1a_K = K;
    M.dg1a_NP = NP;
    M.dg1a_smem = (size_t)2 * T * 2 * K * (AR + NP);
    M.dg1a_AR = AR;
    M.dg1a = true;
}

template <int T>
void launch_dg1a(const Plan& P, const TcPlan& M, const TcCtx& c, cudaStream_t s) {
    allow_dyn_smem(reinterpret_cast<const void*>(tc_dg1a_kernel<T>), kMaxDynSmem);
    tc_dg1a_kernel<T><<<M.dg1a_ntiles, D1_THREADS, M.dg1a_smem, s>>>(
        c, static_cast<const D1Item*>(M.dg1a_items.p), static_cast<const D1Tile*>(M.dg1a_tiles.p), M.dg1a_K,
        M.dg1a_NP, M.dg1a_AR, 2 * M.dg1a_NP, P.n_phi);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

// The stacked-term form of DG1a (MODE CAT_DG1A) or DG1b (CAT_DG1B) when the stacked N
// (2 T r8(rank)) fits one MMA and both operands fit shared memory; TFMM_TC_CAT=0 keeps
// the other forms (for comparisons), as does a DG1a pair count set by the tuning.
template <class VOff, class MOff>
void plan_cat(const Plan& P, TcPlan& M, int mode, bf16* Vb, VOff voff, bf16* Mb, MOff moff) {
    CatPlan& C = mode == CAT_DG1A ? M.cat1a : M.cat1b;
    C.on = false;
    if (const char* e = std::getenv("TFMM_TC_CAT"); e && e[0] == '0') return;
    if (mode == CAT_DG1A && (P.tc_dg1a_pairs != 0 || !fused_enabled())) return;
    const int T = M.T, R = M.R, nt = P.n_theta, np = P.n_phi;
    const int K = mode == CAT_DG1A ? nt : np, K16 = (K + 15) & ~15;
    const int n8max = (int)r8(P.max_rank[mode == CAT_DG1A ? 0 : 1]);
    if (2 * T * n8max > 256) return;
    if (mode == CAT_DG1A && TBM * (K16 / 8) > 4 * CAT_THREADS) return;
    const size_t sbo = (size_t)K16 * 16;
    const size_t smem = (size_t)2 * T * (TBM / 8) * sbo + (size_t)2 * (2 * T * n8max / 8) * sbo;
    if (smem > kMaxDynSmem) return;
    std::vector<CatItem> items(P.items.size());
    std::vector<D1Tile> tiles;
    for (size_t q = 0; q < P.items.size(); ++q) {
        const TuckerItem& d = P.items[q];
        CatItem& it = items[q];
        it.g = d.g; it.alpha = d.alpha; it.rt = d.rt;
        if (mode == CAT_DG1A) {
            it.fac = P.d_factors + d.uth; it.rank = d.rt; it.M = np * R;
            it.a = nullptr; it.a_ld = 0; it.a_ps = 0;
            it.out = Vb + voff((int)q); it.o_ld = r8(np); it.o_ps = (int64_t)d.rt * R * r8(np);
        } else {
            it.fac = P.d_factors + d.uphi; it.rank = d.rp; it.M = d.rt * R;
            it.a = Vb + voff((int)q); it.a_ld = r8(np); it.a_ps = (int64_t)d.rt * R * r8(np);
            const int64_t ldh = r8((int64_t)d.rt * d.rp);
            it.out = Mb + moff((int)q); it.o_ld = ldh; it.o_ps = (int64_t)R * ldh;
        }
        for (int p0 = 0; p0 < it.M; p0 += TBM) tiles.push_back(D1Tile{(int)q, p0});
    }
    TFMM_CUDA_CHECK(device_malloc(&C.items.p, sizeof(CatItem) * items.size()));
    TFMM_CUDA_CHECK(device_malloc(&C.tiles.p, sizeof(D1Tile) * tiles.size()));
    TFMM_CUDA_CHECK(cudaMemcpy(C.items.p, items.data(), sizeof(CatItem) * items.size(), cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(cudaMemcpy(C.tiles.p, tiles.data(), sizeof(D1Tile) * tiles.size(), cudaMemcpyHostToDevice));
    C.ntiles = (int)tiles.size();
    C.K = K;
    C.K16 = K16;
    C.n8max = n8max;
    C.smem = smem;
    C.tcols = 32;
    while (C.tcols < 2 * T * n8max) C.tcols *= 2;
    C.on = true;
}

template <int T, int MODE>
void launch_cat(const Plan& P, const CatPlan& C, const TcCtx& c, cudaStream_t s) {
    allow_dyn_smem(reinterpret_cast<const void*>(tc_cat_kernel<T, MODE>), kMaxDynSmem);
    tc_cat_kernel<T, MODE><<<C.ntiles, CAT_THREADS, C.smem, s>>>(c, static_cast<const CatItem*>(C.items.p),
                                                               static_cast<const D1Tile*>(C.tiles.p), C.K, C.K16,
                                                               C.n8max, C.tcols, P.n_phi);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

}  // namespace

TcPlan* get_tc_plan(Plan& P, int R, int T, cudaStream_t s) {
    build_tc_factors(P, T, s);
    for (auto& m : P.tc)
        if (m->R == R && m->T == T) return m.get();
    auto tp = std::make_unique<TcPlan>();
    TcPlan& M = *tp;
    M.R = R;
    M.T = T;
    const int nt = P.n_theta, np = P.n_phi;
    const int nI = P.G * 2;
    const bf16* F = reinterpret_cast<const bf16*>(P.tc_fac[T].p);
    const std::vector<TcItem>& tci = P.tc_items[T];
    // scratch planes: X (per group), T/S, M'/H, V''/P'', G' (per item)
    enum { BX, BT, BM, BV, BG, NB };
    int64_t sz[NB] = {0, 0, 0, 0, 0};
    struct Off { int64_t x, t, m, v, g; int64_t ldt, ldm, ldv, ldg, ldx; };
    std::vector<Off> of(nI);
    for (int q = 0; q < nI; ++q) {
        const TuckerItem& d = P.items[q];
        const int m = d.rt * d.rp;
        Off& o = of[q];
        o.ldx = r8(d.n_beta);
        if (d.alpha == 0) { o.x = sz[BX]; sz[BX] += (int64_t)2 * T * R * o.ldx; }
        else o.x = of[q - 1].x;
        // T ([r][c]) and S ([r][c]) share a buffer
        o.ldt = r8(d.rb); o.t = sz[BT]; sz[BT] += (int64_t)2 * T * R * o.ldt;
        // M' ([a + r_t r][b]) and H ([r][a + r_t b]) share a buffer
        o.ldm = std::max(r8(d.rp), r8(m));
        o.m = sz[BM]; sz[BM] += (int64_t)2 * T * std::max<int64_t>((int64_t)d.rt * R * r8(d.rp), (int64_t)R * r8(m));
        // V'' ([i_phi + n_phi r][a]) and P'' ([a + r_t r][i_phi]) share a buffer
        o.v = sz[BV]; sz[BV] += (int64_t)2 * T * std::max<int64_t>((int64_t)np * R * r8(d.rt), (int64_t)d.rt * R * r8(np));
        o.ldg = r8(nt); o.g = sz[BG]; sz[BG] += (int64_t)2 * T * np * R * o.ldg;
        for (int b = 0; b < NB; ++b) sz[b] = (sz[b] + 63) & ~int64_t(63);
    }
    for (int b = 0; b < NB; ++b) {
        TFMM_CUDA_CHECK(device_malloc(&M.buf[b], sizeof(bf16) * std::max<int64_t>(sz[b], 1)));
        TFMM_CUDA_CHECK(cudaMemset(M.buf[b], 0, sizeof(bf16) * std::max<int64_t>(sz[b], 1)));
    }
    bf16* X = reinterpret_cast<bf16*>(M.buf[BX]);
    bf16* Tb = reinterpret_cast<bf16*>(M.buf[BT]);
    bf16* Mb = reinterpret_cast<bf16*>(M.buf[BM]);
    bf16* Vb = reinterpret_cast<bf16*>(M.buf[BV]);
    bf16* Gb = reinterpret_cast<bf16*>(M.buf[BG]);
    std::vector<TcProb> pr[8];
    std::vector<MrTile> tl[8];
    for (int q = 0; q < nI; ++q) {
        const TuckerItem& d = P.items[q];
        const TcItem& f = tci[q];
        const Off& o = of[q];
        const int m = d.rt * d.rp;
        TcProb b{};
        b.g = d.g; b.alpha = d.alpha; b.rt = d.rt; b.n_phi = np; b.rwg = d.rwg;
        auto mat = [&](const TcMat& t, const bf16*& ptr, int64_t& ld, int64_t& ps) {
            ptr = F + t.off; ld = t.ld; ps = (int64_t)t.rows * t.ld;
        };
        // AG1: T^T = U_beta^T X_g ; out T planes [r][c]
        TcProb p = b;
        p.M = d.rb; p.N = R; p.K0 = d.n_beta; p.BN = bn_of(R);
        mat(f.ubT, p.A0, p.a_ld0, p.a_ps0);
        p.B0 = X + o.x; p.b_ld0 = o.ldx; p.b_ps0 = (int64_t)R * o.ldx;
        p.out = Tb + o.t; p.o_ld = o.ldt; p.o_ps = (int64_t)R * o.ldt;
        add_tc_tiles(tl[TAG1], (int)pr[TAG1].size(), p.M, p.N); pr[TAG1].push_back(p);
        // AG2: M = C_(3)^T T ; out M' planes [a + r_t r][b]
        p = b;
        p.M = m; p.N = R; p.K0 = d.rb; p.BN = bn_of(R);
        mat(f.c3T, p.A0, p.a_ld0, p.a_ps0);
        p.B0 = Tb + o.t; p.b_ld0 = o.ldt; p.b_ps0 = (int64_t)R * o.ldt;
        p.out = Mb + o.m; p.o_ld = r8(d.rp); p.o_ps = (int64_t)d.rt * R * r8(d.rp);
        add_tc_tiles(tl[TAG2], (int)pr[TAG2].size(), p.M, p.N); pr[TAG2].push_back(p);
        // AG3: V' = M' U_phi^T ; out V'' planes [i_phi + n_phi r][a]
        p = b;
        p.M = d.rt * R; p.N = np; p.K0 = d.rp; p.BN = bn_of(np);
        p.A0 = Mb + o.m; p.a_ld0 = r8(d.rp); p.a_ps0 = (int64_t)d.rt * R * r8(d.rp);
        mat(f.uphT, p.B0, p.b_ld0, p.b_ps0);
        p.out = Vb + o.v; p.o_ld = r8(d.rt); p.o_ps = (int64_t)np * R * r8(d.rt);
        add_tc_tiles(tl[TAG3], (int)pr[TAG3].size(), p.M, p.N); pr[TAG3].push_back(p);
        // AG4: F' = V'' U_theta^T ; out spectra (set at launch)
        p = b;
        p.M = np * R; p.N = nt; p.K0 = d.rt; p.BN = bn_of(nt);
        p.A0 = Vb + o.v; p.a_ld0 = r8(d.rt); p.a_ps0 = (int64_t)np * R * r8(d.rt);
        mat(f.uthT, p.B0, p.b_ld0, p.b_ps0);
        add_tc_tiles(tl[TAG4], (int)pr[TAG4].size(), p.M, p.N); pr[TAG4].push_back(p);
        // DG1a: P' = G' U_theta ; out P'' planes [a + r_t r][i_phi]
        p = b;
        p.M = np * R; p.N = d.rt; p.K0 = nt; p.BN = bn_of(d.rt);
        p.A0 = Gb + o.g; p.a_ld0 = o.ldg; p.a_ps0 = (int64_t)np * R * o.ldg;
        mat(f.uth, p.B0, p.b_ld0, p.b_ps0);
        p.out = Vb + o.v; p.o_ld = r8(np); p.o_ps = (int64_t)d.rt * R * r8(np);
        add_tc_tiles(tl[TDG1A], (int)pr[TDG1A].size(), p.M, p.N); pr[TDG1A].push_back(p);
        // DG1b: H' = P'' U_phi ; out H planes [r][a + r_t b]
        p = b;
        p.M = d.rt * R; p.N = d.rp; p.K0 = np; p.BN = bn_of(d.rp);
        p.A0 = Vb + o.v; p.a_ld0 = r8(np); p.a_ps0 = (int64_t)d.rt * R * r8(np);
        mat(f.uph, p.B0, p.b_ld0, p.b_ps0);
        p.out = Mb + o.m; p.o_ld = r8(m); p.o_ps = (int64_t)R * r8(m);
        add_tc_tiles(tl[TDG1B], (int)pr[TDG1B].size(), p.M, p.N); pr[TDG1B].push_back(p);
        // DG2: S = C_(3) H ; out S planes [r][c]
        p = b;
        p.M = d.rb; p.N = R; p.K0 = m; p.BN = bn_of(R);
        mat(f.c3, p.A0, p.a_ld0, p.a_ps0);
        p.B0 = Mb + o.m; p.b_ld0 = r8(m); p.b_ps0 = (int64_t)R * r8(m);
        p.out = Tb + o.t; p.o_ld = o.ldt; p.o_ps = (int64_t)R * o.ldt;
        add_tc_tiles(tl[TDG2], (int)pr[TDG2].size(), p.M, p.N); pr[TDG2].push_back(p);
    }
    for (int g = 0; g < P.G; ++g) {
        const TuckerItem& d0 = P.items[2 * g];
        const TuckerItem& d1 = P.items[2 * g + 1];
        TcProb p{};
        p.g = g; p.rwg = d0.rwg;
        p.M = d0.n_beta; p.N = R; p.K0 = d0.rb; p.K1 = d1.rb; p.BN = bn_of(R);
        const TcMat& u0 = tci[2 * g].ub;
        const TcMat& u1 = tci[2 * g + 1].ub;
        p.A0 = F + u0.off; p.a_ld0 = u0.ld; p.a_ps0 = (int64_t)u0.rows * u0.ld;
        p.A1 = F + u1.off; p.a_ld1 = u1.ld; p.a_ps1 = (int64_t)u1.rows * u1.ld;
        p.B0 = Tb + of[2 * g].t; p.b_ld0 = of[2 * g].ldt; p.b_ps0 = (int64_t)R * of[2 * g].ldt;
        p.B1 = Tb + of[2 * g + 1].t; p.b_ld1 = of[2 * g + 1].ldt; p.b_ps1 = (int64_t)R * of[2 * g + 1].ldt;
        add_tc_tiles(tl[TDG3], (int)pr[TDG3].size(), p.M, p.N); pr[TDG3].push_back(p);
    }
    for (int st = 0; st < 8; ++st) {
        upload_tc_stage(M.st[st], pr[st], tl[st]);
        if (st == TAG1 || st == TAG2 || st == TDG2 || st == TDG3) build_stage_maps(M.st[st], pr[st], T);
    }
    M.m_off.resize(nI);
    M.v_off.resize(nI);
    for (int q = 0; q < nI; ++q) {
        M.m_off[q] = of[q].m;
        M.v_off[q] = of[q].v;
    }
    plan_fused34(P, M, F, tci, Mb, [&](int q) { return M.m_off[q]; });
    const auto voff = [&](int q) { return M.v_off[q]; };
    const auto moff = [&](int q) { return M.m_off[q]; };
    plan_cat(P, M, CAT_DG1A, Vb, voff, Mb, moff);
    if (!M.cat1a.on) plan_dg1a(P, M, F, tci, Vb, voff);
    plan_cat(P, M, CAT_DG1B, Vb, voff, Mb, moff);
    P.tc.push_back(std::move(tp));
    return P.tc.back().get();
}

void tc_replan_shapes(Plan& P) {
    TFMM_REQUIRE(P.live_graphs == 0, "captured graphs use the current tile lists: destroy them first");
    TFMM_CUDA_CHECK(cudaDeviceSynchronize());  // no launch may still read the old lists
    for (auto& mp : P.tc) {
        TcPlan& M = *mp;
        for (DeviceBuffer* b : {&M.f34_items, &M.f34_tiles, &M.dg1a_items, &M.dg1a_tiles, &M.cat1a.items,
                                &M.cat1a.tiles}) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
        }
        const bf16* F = reinterpret_cast<const bf16*>(P.tc_fac[M.T].p);
        const std::vector<TcItem>& tci = P.tc_items[M.T];
        bf16* Mb = reinterpret_cast<bf16*>(M.buf[2]);
        bf16* Vb = reinterpret_cast<bf16*>(M.buf[3]);
        plan_fused34(P, M, F, tci, Mb, [&](int q) { return M.m_off[q]; });
        const auto voff = [&](int q) { return M.v_off[q]; };
        const auto moff = [&](int q) { return M.m_off[q]; };
        plan_cat(P, M, CAT_DG1A, Vb, voff, Mb, moff);
        M.dg1a = false;
        if (!M.cat1a.on) plan_dg1a(P, M, F, tci, Vb, voff);
    }
}

namespace {

template <int T>
void tc_aggregate_t(Plan& P, TcPlan& M, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    TcCtx c{};
    c.grp_rwg = P.d_grp_rwg; c.R = R; c.G = P.G; c.n_theta = P.n_theta; c.n_dir = P.n_dir; c.err = static_cast<int*>(P.tc_err.p);
    c.spec = spec;
    dim3 gx(64, std::min(P.G * 2, 4096));
    prep_x_kernel<T><<<gx, 256, 0, s>>>(x, ldx, P.d_grp_rwg, reinterpret_cast<const TcProb*>(M.st[TAG1].d_probs),
                                        M.st[TAG1].n_probs, R);
    TFMM_CUDA_CHECK(cudaGetLastError());
    launch_tc<T, TAG1>(M.st[TAG1], c, s);
    launch_tc<T, TAG2>(M.st[TAG2], c, s);
    if (M.fused34) {
        launch_ag34<T>(P, M, c, s);
    } else {
        launch_tc<T, TAG3>(M.st[TAG3], c, s);
        launch_tc<T, TAG4>(M.st[TAG4], c, s);
    }
}

template <int T>
void tc_disaggregate_t(Plan& P, TcPlan& M, const float2* spec, int R, int weights, float2 beta, float2* y,
                       int64_t ldy, cudaStream_t s) {
    TcCtx c{};
    c.grp_rwg = P.d_grp_rwg; c.R = R; c.G = P.G; c.n_theta = P.n_theta; c.n_dir = P.n_dir; c.err = static_cast<int*>(P.tc_err.p);
    c.ld = ldy; c.beta = beta;
    c.y = y;
    if (fused_enabled()) {  // DG1a reads the FP32 spectra itself
        c.spec_in = spec;
        c.w = weights ? P.d_weights : nullptr;
    } else {
        dim3 gg(64, std::min(P.G * 2, 4096));
        prep_g_kernel<T><<<gg, 256, 0, s>>>(spec, weights ? P.d_weights : nullptr,
                                            reinterpret_cast<const TcProb*>(M.st[TDG1A].d_probs), M.st[TDG1A].n_probs,
                                            R, P.G, P.n_theta, P.n_phi);
        TFMM_CUDA_CHECK(cudaGetLastError());
    }
    if (M.cat1a.on)
        launch_cat<T, CAT_DG1A>(P, M.cat1a, c, s);
    else if (M.dg1a)
        launch_dg1a<T>(P, M, c, s);
    else
        launch_tc<T, TDG1A>(M.st[TDG1A], c, s);
    if (M.cat1b.on)
        launch_cat<T, CAT_DG1B>(P, M.cat1b, c, s);
    else
        launch_tc<T, TDG1B>(M.st[TDG1B], c, s);
    launch_tc<T, TDG2>(M.st[TDG2], c, s);
    launch_tc<T, TDG3>(M.st[TDG3], c, s);
}

}  // namespace

void launch_tc_aggregate(Plan& P, int T, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    TcPlan* M = get_tc_plan(P, R, T, s);
    if (T == 2)
        tc_aggregate_t<2>(P, *M, x, R, ldx, spec, s);
    else
        tc_aggregate_t<3>(P, *M, x, R, ldx, spec, s);
}

void launch_tc_disaggregate(Plan& P, int T, const float2* spec, int R, int weights, float2 beta, float2* y,
                            int64_t ldy, cudaStream_t s) {
    TcPlan* M = get_tc_plan(P, R, T, s);
    if (T == 2)
        tc_disaggregate_t<2>(P, *M, spec, R, weights, beta, y, ldy, s);
    else
        tc_disaggregate_t<3>(P, *M, spec, R, weights, beta, y, ldy, s);
}

}  // namespace tfmm
