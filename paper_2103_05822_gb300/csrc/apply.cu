// Hot path: aggregation and disaggregation from Tucker factors (Figs. 2b, 3b)
// and from the uncompressed tensors (Eqs. 3, 5), FP32 complex on CUDA cores.
//
// Every stage is one persistent launch over all groups: each CTA pulls work
// items (a group and component for aggregation, a whole group for
// disaggregation) from a queue ordered longest-first, so groups with uneven
// n_beta and ranks balance across the SMs.  The queue is a ticket counter in
// global memory that the last CTA to leave resets, so consecutive launches
// (and CUDA-graph replays) need no host-side reset.
//
// Per item the two large operands are streamed once from HBM with 16-byte
// non-caching loads: U_beta (stored as r_beta rows of n_beta, i.e. column c of
// U_beta per row) and the mode-3 matricised core C_(3) (r_beta rows of
// r_theta r_phi).  Two access patterns cover all four contractions with them:
//   rowdot  out[c] = sum_j M[c][j] v[j]   one warp per row, shuffle reduction
//                                         (AG1: t = U_beta^T x, DG2: s = C_(3) vec H)
//   rowaxpy out[j] = sum_c M[c][j] s[c]   one thread per column pair
//                                         (AG2: u = t^T C_(3), DG3: U_beta s)
// The small theta / phi factors are staged in shared memory and the r_theta x
// r_phi intermediates never leave the SM.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace tfmm {

namespace {

__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

__host__ __device__ __forceinline__ int64_t round_up_dev(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// acc += a * b (complex)
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}
// acc (two complex) += m (two complex) * s
__device__ __forceinline__ void cfma2(float4& acc, float4 m, float2 s) {
    acc.x = fmaf(m.x, s.x, acc.x);
    acc.x = fmaf(-m.y, s.y, acc.x);
    acc.y = fmaf(m.x, s.y, acc.y);
    acc.y = fmaf(m.y, s.x, acc.y);
    acc.z = fmaf(m.z, s.x, acc.z);
    acc.z = fmaf(-m.w, s.y, acc.z);
    acc.w = fmaf(m.z, s.y, acc.w);
    acc.w = fmaf(m.w, s.x, acc.w);
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Starts pulling the head of an array that a later phase streams into L2, so that
// DRAM stays busy through the short shared-memory phases before it (one thread).
constexpr uint32_t kPrefetchBytes = 128 * 1024;
__device__ __forceinline__ void prefetch_head_l2(const void* p, int64_t bytes) {
    const uint32_t n = (uint32_t)(bytes < (int64_t)kPrefetchBytes ? bytes : (int64_t)kPrefetchBytes) & ~15u;
    if (n) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(n) : "memory");
}

// Next work item of this CTA, or >= n_items when the queue is drained.  The
// CTA that drains last resets the counters for the next launch.
__device__ __forceinline__ int next_item(unsigned* ctr, unsigned* done, int n_items, int* s_item) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ctr, 1u);
        if (t >= (unsigned)n_items) {
            __threadfence();
            const unsigned d = atomicAdd(done, 1u);
            if (d == gridDim.x - 1) {
                atomicExch(ctr, 0u);
                atomicExch(done, 0u);
            }
        }
        *s_item = (int)min(t, (unsigned)n_items);
    }
    __syncthreads();
    return *s_item;
}

// out[c] = sum_j M[c][j] v[j] (CONJ: conj(M)); rows of ld2 float4 (2 complex each)
template <bool CONJ, class Emit>
__device__ __forceinline__ void rowdot(const float4* __restrict__ M, int ld2, int nrows, const float4* v, Emit emit) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < nrows; c += nw) {
        const float4* row = M + (int64_t)c * ld2;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int j = lane; j < ld2; j += 32) {
            const float4 m = ld_stream(row + j);
            const float4 x = v[j];
            if (CONJ) {
                cfma_conj(a0, make_float2(m.x, m.y), make_float2(x.x, x.y));
                cfma_conj(a1, make_float2(m.z, m.w), make_float2(x.z, x.w));
            } else {
                cfma(a0, make_float2(m.x, m.y), make_float2(x.x, x.y));
                cfma(a1, make_float2(m.z, m.w), make_float2(x.z, x.w));
            }
        }
        float2 s = warp_sum(make_float2(a0.x + a1.x, a0.y + a1.y));
        if (lane == 0) emit(c, s);
    }
}

// out[j] (float4 = two complex columns) = sum_c M[c][j] s[c]; `part` holds
// blockDim float4 of scratch for the split-row case.
template <class Emit>
__device__ __forceinline__ void rowaxpy(const float4* __restrict__ M, int ld2, int nrows, const float2* s,
                                        float4* part, Emit emit) {
    const int NT = blockDim.x, tid = threadIdx.x;
    if (2 * ld2 >= NT) {
        for (int j = tid; j < ld2; j += NT) {
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
            int c = 0;
#pragma unroll 4
            for (; c + 1 < nrows; c += 2) {
                const float4 m0 = ld_stream(M + (int64_t)c * ld2 + j);
                const float4 m1 = ld_stream(M + (int64_t)(c + 1) * ld2 + j);
                cfma2(a0, m0, s[c]);
                cfma2(a1, m1, s[c + 1]);
            }
            if (c < nrows) cfma2(a0, ld_stream(M + (int64_t)c * ld2 + j), s[c]);
            emit(j, add4(a0, a1));
        }
    } else {
        const int S = NT / ld2;  // >= 2 slices of rows
        const int j = tid % ld2, sl = tid / ld2;
        if (sl < S) {
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int c = sl; c < nrows; c += S) cfma2(a0, ld_stream(M + (int64_t)c * ld2 + j), s[c]);
            part[sl * ld2 + j] = a0;
        }
        __syncthreads();
        for (int jj = tid; jj < ld2; jj += NT) {
            float4 a = part[jj];
            for (int q = 1; q < S; ++q) a = add4(a, part[q * ld2 + jj]);
            emit(jj, a);
        }
    }
}

// C(m, n) = sum_{k < K} A(m, k) B(k, n) for the small theta / phi contractions, all
// operands in shared memory: every thread computes a TM x TN block of outputs in
// registers, so a complex multiply-add costs (TM + TN) / (TM TN) shared-memory loads
// instead of two.  a(m, k) and b(k, n) read the operands (indices clamped to the
// valid range); emit(m, n, v) stores one result.
template <int TM, int TN, class LA, class LB, class Emit>
__device__ __forceinline__ void smem_gemm(int M, int N, int K, LA a, LB b, Emit emit) {
    const int mt = (M + TM - 1) / TM, nt = (N + TN - 1) / TN;
    for (int t = threadIdx.x; t < mt * nt; t += blockDim.x) {
        const int m0 = (t % mt) * TM, n0 = (t / mt) * TN;
        float2 acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
        int mi[TM], nj[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) mi[i] = min(m0 + i, M - 1);
#pragma unroll
        for (int j = 0; j < TN; ++j) nj[j] = min(n0 + j, N - 1);
        for (int k = 0; k < K; ++k) {
            float2 av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = a(mi[i], k);
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = b(k, nj[j]);
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) cfma(acc[i][j], av[i], bv[j]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (m0 + i < M && n0 + j < N) emit(m0 + i, n0 + j, acc[i][j]);
    }
}

struct SmemLayout {  // offsets in float2 units, each 16-byte aligned
    int o_a, o_b, o_c, o_d, o_e, o_f, o_g, o_h, total;
    int ldt, ldp, ldv, ldg;
};

struct AggArgs {
    const TuckerItem* items;
    const int* order;
    int n_items;
    const float2* fac;
    const int* grp_rwg;
    const float2* x;
    int64_t ldx;
    float2* spec;
    int n_theta, n_phi, n_dir, G, R;
    unsigned* ctr;
    unsigned* done;
    SmemLayout L;
};

// Aggregation (Fig. 2b) of one (group, alpha) per work item.  SVD: the plan holds
// the truncated SVD of the aggregation matrix (Sec. II.C comparator) as a Tucker
// format with identity theta / phi factors, core C_(3) = (U Sigma)^T and U_beta =
// conj(V): the spectrum is AG1 followed by AG2 written straight to it.
template <bool SVD>
__global__ void __launch_bounds__(512, 3) tucker_aggregate_kernel(const AggArgs a) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    __shared__ int s_item;
    float2* s_ut = sm + a.L.o_a;   // U_theta, ld ldt
    float2* s_up = sm + a.L.o_b;   // U_phi, ld ldp
    float2* s_x = sm + a.L.o_c;    // x_g (padded to ld_nb); later V (ld ldv)
    float2* s_V = s_x;
    float2* s_t = sm + a.L.o_d;    // t = U_beta^T x_g
    float2* s_M = sm + a.L.o_e;    // M[a + r_t b]
    float4* s_part = reinterpret_cast<float4*>(sm + a.L.o_f);
    const int NT = blockDim.x, tid = threadIdx.x;
    for (;;) {
        const int q = next_item(a.ctr, a.done, a.n_items, &s_item);
        if (q >= a.n_items) break;
        const TuckerItem d = a.items[a.order[q]];
        const float2* Ub = a.fac + d.ub;
        const float2* Cc = a.fac + d.core;
        const float2* Up = a.fac + d.uphi;
        const float2* Ut = a.fac + d.uth;
        if (tid == 0) {  // AG1 and AG2 stream these right after the staging below
            prefetch_head_l2(Ub, (int64_t)d.rb * d.ld_nb * 8);
            prefetch_head_l2(Cc, (int64_t)d.rb * d.ld_ab * 8);
        }
        for (int r = 0; r < a.R; ++r) {
            // stage the small factors and the group's currents
            if (!SVD) {
                for (int e = tid; e < a.n_theta * d.rt; e += NT) s_ut[(e % a.n_theta) + a.L.ldt * (e / a.n_theta)] = Ut[e];
                for (int e = tid; e < a.n_phi * d.rp; e += NT) s_up[(e % a.n_phi) + a.L.ldp * (e / a.n_phi)] = Up[e];
            }
            for (int n = tid; n < d.ld_nb; n += NT)
                s_x[n] = n < d.n_beta ? a.x[(int64_t)a.grp_rwg[d.rwg + n] + a.ldx * r] : make_float2(0.f, 0.f);
            __syncthreads();
            // AG1: t[c] = sum_n U_beta[n, c] x_n
            rowdot<false>(reinterpret_cast<const float4*>(Ub), d.ld_nb / 2, d.rb, reinterpret_cast<const float4*>(s_x),
                          [&](int c, float2 v) { s_t[c] = v; });
            __syncthreads();
            if (SVD) {
                // F[i] = sum_c B[i, c] t[c], i = i_theta + n_theta i_phi (the core's column index)
                float2* out = a.spec + (((int64_t)r * a.G + d.g) * 2 + d.alpha) * a.n_dir;
                rowaxpy(reinterpret_cast<const float4*>(Cc), d.ld_ab / 2, d.rb, s_t, s_part, [&](int j, float4 v) {
                    out[2 * j] = make_float2(v.x, v.y);
                    if (2 * j + 1 < a.n_dir) out[2 * j + 1] = make_float2(v.z, v.w);
                });
                __syncthreads();
                continue;
            }
            // AG2: M[ab] = sum_c C_(3)[c, ab] t[c]
            rowaxpy(reinterpret_cast<const float4*>(Cc), d.ld_ab / 2, d.rb, s_t, s_part,
                    [&](int j, float4 v) { reinterpret_cast<float4*>(s_M)[j] = v; });
            __syncthreads();
            // AG3: V[i_phi, a] = sum_b U_phi[i_phi, b] M[a, b]
            {
                const int ldp = a.L.ldp, ldv = a.L.ldv, rt = d.rt;
                smem_gemm<2, 2>(a.n_phi, rt, d.rp, [&](int ip, int b) { return s_up[ip + ldp * b]; },
                                [&](int b, int aa) { return s_M[aa + rt * b]; },
                                [&](int ip, int aa, float2 v) { s_V[ip + ldv * aa] = v; });
            }
            __syncthreads();
            // AG4: F[i_theta, i_phi] = sum_a U_theta[i_theta, a] V[i_phi, a]
            {
                float2* out = a.spec + (((int64_t)r * a.G + d.g) * 2 + d.alpha) * a.n_dir;
                const int ldt = a.L.ldt, ldv = a.L.ldv, nth = a.n_theta;
                smem_gemm<2, 4>(nth, a.n_phi, d.rt, [&](int it, int aa) { return s_ut[it + ldt * aa]; },
                                [&](int aa, int ip) { return s_V[ip + ldv * aa]; },
                                [&](int it, int ip, float2 v) { out[it + nth * ip] = v; });
            }
            __syncthreads();
        }
    }
}

struct DisArgs {
    const TuckerItem* items;
    const int* order;  // group ids, longest first
    int n_items;       // groups
    const float2* fac;
    const int* grp_rwg;
    const float2* spec;
    const float* w;    // n_dir weights or null
    float2* y;
    int64_t ldy;
    float2 beta;
    int n_theta, n_phi, n_dir, G, R;
    unsigned* ctr;
    unsigned* done;
    SmemLayout L;
};

// Disaggregation (Fig. 3b) of one group (both alpha) per work item.  SVD (see the
// aggregation): H is conj(W g) itself, then DG2 and DG3.
template <bool SVD>
__global__ void __launch_bounds__(512, 3) tucker_disaggregate_kernel(const DisArgs a) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    __shared__ int s_item;
    float2* s_ut = sm + a.L.o_a;
    float2* s_up = sm + a.L.o_b;
    float4* s_y4 = reinterpret_cast<float4*>(sm + a.L.o_c);  // accumulated y_g (ld_nb)
    float2* s_y = sm + a.L.o_c;
    float2* s_H = sm + a.L.o_d;   // H (ld_ab, padded with zeros)
    float2* s_s = sm + a.L.o_e;   // s = C_(3) vec(H)
    float2* s_G = sm + a.L.o_f;   // conj(W g) (ld ldg); aliased by the rowaxpy scratch
    float4* s_part = reinterpret_cast<float4*>(sm + a.L.o_f);
    float2* s_P = sm + a.L.o_g;   // P[a + r_t i_phi]
    const int NT = blockDim.x, tid = threadIdx.x;
    for (;;) {
        const int q = next_item(a.ctr, a.done, a.n_items, &s_item);
        if (q >= a.n_items) break;
        const int g = a.order[q];
        for (int r = 0; r < a.R; ++r) {
            const TuckerItem d0 = a.items[2 * g];
            for (int n = tid; n < d0.ld_nb; n += NT) s_y[n] = make_float2(0.f, 0.f);
            for (int al = 0; al < 2; ++al) {
                const TuckerItem d = a.items[2 * g + al];
                const float2* Ub = a.fac + d.ub;
                const float2* Cc = a.fac + d.core;
                const float2* Up = a.fac + d.uphi;
                const float2* Ut = a.fac + d.uth;
                const float2* gin = a.spec + (((int64_t)r * a.G + g) * 2 + al) * a.n_dir;
                if (tid == 0) {  // DG2 and DG3 stream these after the DG1 phase
                    prefetch_head_l2(Cc, (int64_t)d.rb * d.ld_ab * 8);
                    prefetch_head_l2(Ub, (int64_t)d.rb * d.ld_nb * 8);
                }
                if (SVD) {
                    for (int o = tid; o < d.ld_ab; o += NT) {
                        float2 v = make_float2(0.f, 0.f);
                        if (o < a.n_dir) {
                            const float2 gv = gin[o];
                            const float wt = a.w ? a.w[o] : 1.0f;
                            v = make_float2(wt * gv.x, -wt * gv.y);
                        }
                        s_H[o] = v;
                    }
                    __syncthreads();
                } else {
                for (int e = tid; e < a.n_theta * d.rt; e += NT) s_ut[(e % a.n_theta) + a.L.ldt * (e / a.n_theta)] = Ut[e];
                for (int e = tid; e < a.n_phi * d.rp; e += NT) s_up[(e % a.n_phi) + a.L.ldp * (e / a.n_phi)] = Up[e];
                for (int o = tid; o < a.n_dir; o += NT) {
                    float2 v = gin[o];
                    const float wt = a.w ? a.w[o] : 1.0f;
                    s_G[(o % a.n_theta) + a.L.ldg * (o / a.n_theta)] = make_float2(wt * v.x, -wt * v.y);
                }
                __syncthreads();
                // DG1: P = U_theta^T conj(W g), then H = P U_phi
                {
                    const int ldt = a.L.ldt, ldg = a.L.ldg, ldp = a.L.ldp, rt = d.rt;
                    smem_gemm<2, 4>(rt, a.n_phi, a.n_theta, [&](int aa, int it) { return s_ut[it + ldt * aa]; },
                                    [&](int it, int ip) { return s_G[it + ldg * ip]; },
                                    [&](int aa, int ip, float2 v) { s_P[aa + rt * ip] = v; });
                    __syncthreads();
                    smem_gemm<2, 2>(rt, d.rp, a.n_phi, [&](int aa, int ip) { return s_P[aa + rt * ip]; },
                                    [&](int ip, int b) { return s_up[ip + ldp * b]; },
                                    [&](int aa, int b, float2 v) { s_H[aa + rt * b] = v; });
                    for (int o = rt * d.rp + tid; o < d.ld_ab; o += NT) s_H[o] = make_float2(0.f, 0.f);
                }
                __syncthreads();
                }
                // DG2: s[c] = sum_ab C_(3)[c, ab] H[ab]
                rowdot<false>(reinterpret_cast<const float4*>(Cc), d.ld_ab / 2, d.rb,
                              reinterpret_cast<const float4*>(s_H), [&](int c, float2 v) { s_s[c] = v; });
                __syncthreads();
                if (tid == 0 && al == 0) {  // the next component's C while this one's U_beta streams
                    const TuckerItem d1 = a.items[2 * g + 1];
                    prefetch_head_l2(a.fac + d1.core, (int64_t)d1.rb * d1.ld_ab * 8);
                }
                // DG3: y_n += conj(sum_c U_beta[n, c] s[c])
                rowaxpy(reinterpret_cast<const float4*>(Ub), d.ld_nb / 2, d.rb, s_s, s_part, [&](int j, float4 v) {
                    float4 o = s_y4[j];
                    s_y4[j] = make_float4(o.x + v.x, o.y - v.y, o.z + v.z, o.w - v.w);
                });
                __syncthreads();
            }
            // y = beta y + y_g
            for (int n = tid; n < d0.n_beta; n += NT) {
                float2* dst = a.y + (int64_t)a.grp_rwg[d0.rwg + n] + a.ldy * r;
                float2 v = s_y[n];
                if (a.beta.x != 0.f || a.beta.y != 0.f) {
                    const float2 old = *dst;
                    v.x += a.beta.x * old.x - a.beta.y * old.y;
                    v.y += a.beta.x * old.y + a.beta.y * old.x;
                }
                *dst = v;
            }
            __syncthreads();
        }
    }
}

struct DenseAggArgs {
    const DenseItem* items;
    const int* order;
    int n_items;
    const float2* A;
    const int* grp_rwg;
    const float2* x;
    int64_t ldx;
    float2* spec;
    int n_dir, ld_dir, G, R;
    int part_off;  // float4 offset of the rowaxpy scratch in shared memory
    unsigned* ctr;
    unsigned* done;
};

// Eq. 3: F = A x_g, one (group, alpha) per work item.
__global__ void __launch_bounds__(512) dense_aggregate_kernel(const DenseAggArgs a) {
    extern __shared__ float4 smem4[];
    float2* s_x = reinterpret_cast<float2*>(smem4);             // n_beta (padded to 16 bytes)
    float4* s_part = smem4 + a.part_off;                         // rowaxpy scratch, blockDim float4
    __shared__ int s_item;
    const int NT = blockDim.x, tid = threadIdx.x;
    for (;;) {
        const int q = next_item(a.ctr, a.done, a.n_items, &s_item);
        if (q >= a.n_items) break;
        const DenseItem d = a.items[a.order[q]];
        for (int r = 0; r < a.R; ++r) {
            for (int n = tid; n < d.n_beta; n += NT) s_x[n] = a.x[(int64_t)a.grp_rwg[d.rwg + n] + a.ldx * r];
            __syncthreads();
            float2* out = a.spec + (((int64_t)r * a.G + d.g) * 2 + d.alpha) * a.n_dir;
            const int ld2 = a.ld_dir / 2;
            rowaxpy(reinterpret_cast<const float4*>(a.A + d.a), ld2, d.n_beta, s_x, s_part, [&](int j, float4 v) {
                out[2 * j] = make_float2(v.x, v.y);
                if (2 * j + 1 < a.n_dir) out[2 * j + 1] = make_float2(v.z, v.w);
            });
            __syncthreads();
        }
    }
}

struct DenseDisArgs {
    const DenseItem* items;
    const int* order;
    int n_items;
    const float2* A;
    const int* grp_rwg;
    const float2* spec;
    const float* w;
    float2* y;
    int64_t ldy;
    float2 beta;
    int n_dir, ld_dir, G, R;
    unsigned* ctr;
    unsigned* done;
};

// Eq. 5: y_g = beta y_g + sum_alpha A_alpha^H (W g_alpha), one group per work item.
__global__ void __launch_bounds__(512) dense_disaggregate_kernel(const DenseDisArgs a) {
    extern __shared__ float4 smem4[];
    float2* s_g = reinterpret_cast<float2*>(smem4);  // ld_dir
    float2* s_y = s_g + a.ld_dir;                    // n_beta
    __shared__ int s_item;
    const int NT = blockDim.x, tid = threadIdx.x;
    for (;;) {
        const int q = next_item(a.ctr, a.done, a.n_items, &s_item);
        if (q >= a.n_items) break;
        const int g = a.order[q];
        for (int r = 0; r < a.R; ++r) {
            const DenseItem d0 = a.items[2 * g];
            for (int al = 0; al < 2; ++al) {
                const DenseItem d = a.items[2 * g + al];
                const float2* gin = a.spec + (((int64_t)r * a.G + g) * 2 + al) * a.n_dir;
                for (int o = tid; o < a.ld_dir; o += NT) {
                    const float wt = (o < a.n_dir) ? (a.w ? a.w[o] : 1.0f) : 0.0f;
                    const float2 v = (o < a.n_dir) ? gin[o] : make_float2(0.f, 0.f);
                    s_g[o] = make_float2(wt * v.x, wt * v.y);
                }
                __syncthreads();
                rowdot<true>(reinterpret_cast<const float4*>(a.A + d.a), a.ld_dir / 2, d.n_beta,
                             reinterpret_cast<const float4*>(s_g), [&](int n, float2 v) {
                                 if (al == 0) {
                                     s_y[n] = v;
                                 } else {
                                     s_y[n].x += v.x;
                                     s_y[n].y += v.y;
                                 }
                             });
                __syncthreads();
            }
            for (int n = tid; n < d0.n_beta; n += NT) {
                float2* dst = a.y + (int64_t)a.grp_rwg[d0.rwg + n] + a.ldy * r;
                float2 v = s_y[n];
                if (a.beta.x != 0.f || a.beta.y != 0.f) {
                    const float2 old = *dst;
                    v.x += a.beta.x * old.x - a.beta.y * old.y;
                    v.y += a.beta.x * old.y + a.beta.y * old.x;
                }
                *dst = v;
            }
            __syncthreads();
        }
    }
}

__global__ void to_f32_pad_kernel(const double2* __restrict__ in, int64_t n, int64_t m, int64_t ldi,
                                  float2* __restrict__ out, int64_t ldo) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const double2 v = in[i + ldi * j];
        out[i + ldo * j] = make_float2((float)v.x, (float)v.y);
    }
}

int grid1d(int64_t total, int threads = 256) {
    int64_t b = (total + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8));
}

int odd_ld(int n) { return (n % 2 == 0) ? n + 1 : n; }

int al16(int v) { return (v + 1) / 2 * 2; }  // float2 count rounded to 16 bytes

SmemLayout agg_layout(const Plan& P, int NT) {
    SmemLayout L{};
    L.ldt = odd_ld(P.n_theta);
    L.ldp = odd_ld(P.n_phi);
    L.ldv = odd_ld(P.n_phi);
    int o = 0;
    L.o_a = o; o += al16(L.ldt * P.max_rank[0]);
    L.o_b = o; o += al16(L.ldp * P.max_rank[1]);
    L.o_c = o; o += al16(std::max(P.max_ldnb, L.ldv * P.max_rank[0]));
    L.o_d = o; o += al16(P.max_rank[2]);
    L.o_e = o; o += al16(P.max_ldab);
    L.o_f = o; o += 2 * NT;  // rowaxpy scratch: NT float4
    L.total = o;
    return L;
}

// SVD plans: x (or y), t (or s), the core row buffer H (N_dir, disaggregation) and the
// rowaxpy scratch; no theta / phi factors are staged.
SmemLayout svd_agg_layout(const Plan& P, int NT) {
    SmemLayout L{};
    int o = 0;
    L.o_a = L.o_b = L.o_e = 0;
    L.o_c = o; o += al16(P.max_ldnb);
    L.o_d = o; o += al16(P.max_rank[2]);
    L.o_f = o; o += 2 * NT;
    L.total = o;
    return L;
}

SmemLayout svd_dis_layout(const Plan& P, int NT) {
    SmemLayout L{};
    int o = 0;
    L.o_a = L.o_b = L.o_g = 0;
    L.o_c = o; o += al16(P.max_ldnb);
    L.o_d = o; o += al16(P.max_ldab);
    L.o_e = o; o += al16(P.max_rank[2]);
    L.o_f = o; o += 2 * NT;
    L.total = o;
    return L;
}

SmemLayout dis_layout(const Plan& P, int NT) {
    SmemLayout L{};
    L.ldt = odd_ld(P.n_theta);
    L.ldp = odd_ld(P.n_phi);
    L.ldg = odd_ld(P.n_theta);
    int o = 0;
    L.o_a = o; o += al16(L.ldt * P.max_rank[0]);
    L.o_b = o; o += al16(L.ldp * P.max_rank[1]);
    L.o_c = o; o += al16(P.max_ldnb);
    L.o_d = o; o += al16(P.max_ldab);
    L.o_e = o; o += al16(P.max_rank[2]);
    L.o_f = o; o += al16(std::max(L.ldg * P.n_phi, 2 * NT));
    L.o_g = o; o += al16(P.max_rank[0] * P.n_phi);
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ split path
// Plans with few, large work items (the trihedral's 19 groups: 38 items for 152 SMs)
// leave most SMs idle with one item per CTA.  The split path runs each stage as three
// launches that spread every item over many CTAs, with the items' intermediates in
// plan-owned scratch (t / s: r_beta, M / H: ld_ab complex per item):
//   aggregation     SA1: t = U_beta^T x_g, blocks of kSplitRows rows per CTA (Fig. 2b step 1)
//                   SA2: M = C_(3)^T t, blocks of kSplitCols column pairs per CTA
//                   SA3: AG3 + AG4 from M, one CTA per item (Fig. 2b steps 2-4)
//   disaggregation  SD1: H = U_theta^T conj(W g) U_phi, one CTA per item (Fig. 3b step 1)
//                   SD2: s = C_(3) vec(H), blocks of rows (step 2)
//                   SD3: y_g = beta y_g + conj(sum_alpha U_beta s), blocks of column pairs of
//                        U_beta^T covering both components of a group (step 3)
constexpr int kSplitRows = 16;  // one row per warp of 512 threads
constexpr int kSplitCols = 64;  // float4 (two complex) columns per CTA: 8 slices of rows

struct SplitTile { int item, start; };  // item (or group for SD3) and first row / column pair

struct SplitArgs {
    const TuckerItem* items;
    const SplitTile* tiles;
    const float2* fac;
    const int* grp_rwg;
    const float2* x;      // SA1
    int64_t ldx;
    const float2* spec;   // SD1 input
    const float* w;       // SD1 weights or null
    float2* spec_out;     // SA3 output
    float2* y;            // SD3 output
    int64_t ldy;
    float2 beta;
    float2* scratch;      // per item: [r_beta slot | ld_ab slot] (offsets in TuckerItem order)
    const int64_t* scr_off;
    int n_theta, n_phi, n_dir, G, r;
    SmemLayout L;
};

// out[j0 + j] = sum_{c < nrows} M[c][j0 + j] s[c] for j < cbv (float4 columns): the CTA
// splits into NT / kSplitCols slices of rows, summed through `part` (NT float4).
template <class Emit>
__device__ __forceinline__ void colblock_axpy(const float4* __restrict__ M, int64_t ld2, int j0, int cbv, int nrows,
                                              const float2* s, float4* part, Emit emit) {
    const int tid = threadIdx.x, S = blockDim.x / kSplitCols;
    const int j = tid % kSplitCols, sl = tid / kSplitCols;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    if (j < cbv && sl < S) {
        const float4* col = M + j0 + j;
        int c = sl;
#pragma unroll 2
        for (; c + S < nrows; c += 2 * S) {
            const float4 m0 = ld_stream(col + (int64_t)c * ld2);
            const float4 m1 = ld_stream(col + (int64_t)(c + S) * ld2);
            cfma2(a0, m0, s[c]);
            cfma2(a1, m1, s[c + S]);
        }
        if (c < nrows) cfma2(a0, ld_stream(col + (int64_t)c * ld2), s[c]);
    }
    if (sl < S) part[sl * kSplitCols + j] = add4(a0, a1);
    __syncthreads();
    for (int jj = tid; jj < cbv; jj += blockDim.x) {
        float4 a = part[jj];
        for (int q = 1; q < S; ++q) a = add4(a, part[q * kSplitCols + jj]);
        emit(j0 + jj, a);
    }
}

// SA1: t[c] = sum_n U_beta[n, c] x_n for the rows c of one tile
__global__ void __launch_bounds__(512) split_ag1_kernel(const SplitArgs a) {
    extern __shared__ float4 smem4[];
    float2* s_x = reinterpret_cast<float2*>(smem4);
    const SplitTile t = a.tiles[blockIdx.x];
    const TuckerItem d = a.items[t.item];
    for (int n = threadIdx.x; n < d.ld_nb; n += blockDim.x)
        s_x[n] = n < d.n_beta ? a.x[(int64_t)a.grp_rwg[d.rwg + n] + a.ldx * a.r] : make_float2(0.f, 0.f);
    __syncthreads();
    float2* tout = a.scratch + a.scr_off[t.item];
    const int rows = min(kSplitRows, d.rb - t.start);
    rowdot<false>(reinterpret_cast<const float4*>(a.fac + d.ub) + (int64_t)t.start * (d.ld_nb / 2), d.ld_nb / 2, rows,
                  reinterpret_cast<const float4*>(s_x), [&](int c, float2 v) { tout[t.start + c] = v; });
}

// SA2: M[ab] = sum_c C_(3)[c, ab] t[c] for the column pairs of one tile
__global__ void __launch_bounds__(512) split_ag2_kernel(const SplitArgs a) {
    extern __shared__ float4 smem4[];
    float4* s_part = smem4;
    float2* s_t = reinterpret_cast<float2*>(smem4 + blockDim.x);
    const SplitTile t = a.tiles[blockIdx.x];
    const TuckerItem d = a.items[t.item];
    const float2* tin = a.scratch + a.scr_off[t.item];
    for (int c = threadIdx.x; c < d.rb; c += blockDim.x) s_t[c] = tin[c];
    __syncthreads();
    float4* mout = reinterpret_cast<float4*>(a.scratch + a.scr_off[t.item] + round_up_dev(d.rb, 2));
    const int ld2 = d.ld_ab / 2;
    colblock_axpy(reinterpret_cast<const float4*>(a.fac + d.core), ld2, t.start, min(kSplitCols, ld2 - t.start), d.rb,
                  s_t, s_part, [&](int j, float4 v) { mout[j] = v; });
}

// SA3: AG3 + AG4 of one item from its M (one CTA per item)
__global__ void __launch_bounds__(512) split_ag34_kernel(const SplitArgs a) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    float2* s_ut = sm + a.L.o_a;
    float2* s_up = sm + a.L.o_b;
    float2* s_V = sm + a.L.o_c;
    float2* s_M = sm + a.L.o_e;
    const int q = blockIdx.x, NT = blockDim.x, tid = threadIdx.x;
    const TuckerItem d = a.items[q];
    const float2* Ut = a.fac + d.uth;
    const float2* Up = a.fac + d.uphi;
    const float2* min_ = a.scratch + a.scr_off[q] + round_up_dev(d.rb, 2);
    for (int e = tid; e < a.n_theta * d.rt; e += NT) s_ut[(e % a.n_theta) + a.L.ldt * (e / a.n_theta)] = Ut[e];
    for (int e = tid; e < a.n_phi * d.rp; e += NT) s_up[(e % a.n_phi) + a.L.ldp * (e / a.n_phi)] = Up[e];
    for (int e = tid; e < d.rt * d.rp; e += NT) s_M[e] = min_[e];
    __syncthreads();
    {
        const int ldp = a.L.ldp, ldv = a.L.ldv, rt = d.rt;
        smem_gemm<2, 2>(a.n_phi, rt, d.rp, [&](int ip, int b) { return s_up[ip + ldp * b]; },
                        [&](int b, int aa) { return s_M[aa + rt * b]; },
                        [&](int ip, int aa, float2 v) { s_V[ip + ldv * aa] = v; });
    }
    __syncthreads();
    float2* out = a.spec_out + (((int64_t)a.r * a.G + d.g) * 2 + d.alpha) * a.n_dir;
    const int ldt = a.L.ldt, ldv = a.L.ldv, nth = a.n_theta;
    smem_gemm<2, 4>(nth, a.n_phi, d.rt, [&](int it, int aa) { return s_ut[it + ldt * aa]; },
                    [&](int aa, int ip) { return s_V[ip + ldv * aa]; },
                    [&](int it, int ip, float2 v) { out[it + nth * ip] = v; });
}

// SD1: H = U_theta^T conj(W g) U_phi of one item (one CTA per item), zero-padded to ld_ab
__global__ void __launch_bounds__(512) split_dg1_kernel(const SplitArgs a) {
    extern __shared__ float4 smem4[];
    float2* sm = reinterpret_cast<float2*>(smem4);
    float2* s_ut = sm + a.L.o_a;
    float2* s_up = sm + a.L.o_b;
    float2* s_G = sm + a.L.o_f;
    float2* s_P = sm + a.L.o_g;
    const int q = blockIdx.x, NT = blockDim.x, tid = threadIdx.x;
    const TuckerItem d = a.items[q];
    const float2* Ut = a.fac + d.uth;
    const float2* Up = a.fac + d.uphi;
    const float2* gin = a.spec + (((int64_t)a.r * a.G + d.g) * 2 + d.alpha) * a.n_dir;
    for (int e = tid; e < a.n_theta * d.rt; e += NT) s_ut[(e % a.n_theta) + a.L.ldt * (e / a.n_theta)] = Ut[e];
    for (int e = tid; e < a.n_phi * d.rp; e += NT) s_up[(e % a.n_phi) + a.L.ldp * (e / a.n_phi)] = Up[e];
    for (int o = tid; o < a.n_dir; o += NT) {
        const float2 v = gin[o];
        const float wt = a.w ? a.w[o] : 1.0f;
        s_G[(o % a.n_theta) + a.L.ldg * (o / a.n_theta)] = make_float2(wt * v.x, -wt * v.y);
    }
    __syncthreads();
    const int ldt = a.L.ldt, ldg = a.L.ldg, ldp = a.L.ldp, rt = d.rt;
    smem_gemm<2, 4>(rt, a.n_phi, a.n_theta, [&](int aa, int it) { return s_ut[it + ldt * aa]; },
                    [&](int it, int ip) { return s_G[it + ldg * ip]; },
                    [&](int aa, int ip, float2 v) { s_P[aa + rt * ip] = v; });
    __syncthreads();
    float2* hout = a.scratch + a.scr_off[q] + round_up_dev(d.rb, 2);
    smem_gemm<2, 2>(rt, d.rp, a.n_phi, [&](int aa, int ip) { return s_P[aa + rt * ip]; },
                    [&](int ip, int b) { return s_up[ip + ldp * b]; },
                    [&](int aa, int b, float2 v) { hout[aa + rt * b] = v; });
    for (int o = rt * d.rp + tid; o < d.ld_ab; o += NT) hout[o] = make_float2(0.f, 0.f);
}

// SD2: s[c] = sum_ab C_(3)[c, ab] H[ab] for the rows c of one tile
__global__ void __launch_bounds__(512) split_dg2_kernel(const SplitArgs a) {
    extern __shared__ float4 smem4[];
    float2* s_H = reinterpret_cast<float2*>(smem4);
    const SplitTile t = a.tiles[blockIdx.x];
    const TuckerItem d = a.items[t.item];
    float2* slot = a.scratch + a.scr_off[t.item];
    const float2* hin = slot + round_up_dev(d.rb, 2);
    for (int o = threadIdx.x; o < d.ld_ab; o += blockDim.x) s_H[o] = hin[o];
    __syncthreads();
    const int rows = min(kSplitRows, d.rb - t.start);
    rowdot<false>(reinterpret_cast<const float4*>(a.fac + d.core) + (int64_t)t.start * (d.ld_ab / 2), d.ld_ab / 2, rows,
                  reinterpret_cast<const float4*>(s_H), [&](int c, float2 v) { slot[t.start + c] = v; });
}

// SD3: y = beta y + conj(U_beta^(0) s^(0) + U_beta^(1) s^(1)) for the column pairs of one
// tile of group t.item (both components)
__global__ void __launch_bounds__(512) split_dg3_kernel(const SplitArgs a) {
    extern __shared__ float4 smem4[];
    float4* s_part = smem4;
    float4* s_acc = smem4 + blockDim.x;
    float2* s_s = reinterpret_cast<float2*>(smem4 + blockDim.x + kSplitCols);
    const SplitTile t = a.tiles[blockIdx.x];
    const int g = t.item;
    const TuckerItem d0 = a.items[2 * g];
    const int ld2 = d0.ld_nb / 2, cbv = min(kSplitCols, ld2 - t.start);
    for (int al = 0; al < 2; ++al) {
        const TuckerItem d = a.items[2 * g + al];
        const float2* sin_ = a.scratch + a.scr_off[2 * g + al];
        for (int c = threadIdx.x; c < d.rb; c += blockDim.x) s_s[c] = sin_[c];
        __syncthreads();
        colblock_axpy(reinterpret_cast<const float4*>(a.fac + d.ub), ld2, t.start, cbv, d.rb, s_s, s_part,
                      [&](int j, float4 v) {
                          const int jj = j - t.start;
                          s_acc[jj] = al == 0 ? v : add4(s_acc[jj], v);
                      });
        __syncthreads();
    }
    for (int jj = threadIdx.x; jj < 2 * cbv; jj += blockDim.x) {
        const int n = 2 * t.start + jj;
        if (n >= d0.n_beta) continue;
        const float4 v4 = s_acc[jj >> 1];
        float2 v = (jj & 1) ? make_float2(v4.z, -v4.w) : make_float2(v4.x, -v4.y);
        float2* dst = a.y + (int64_t)a.grp_rwg[d0.rwg + n] + a.ldy * a.r;
        if (a.beta.x != 0.f || a.beta.y != 0.f) {
            const float2 old = *dst;
            v.x += a.beta.x * old.x - a.beta.y * old.y;
            v.y += a.beta.x * old.y + a.beta.y * old.x;
        }
        *dst = v;
    }
}

template <class K>
Schedule make_schedule(K kernel, int NT, size_t smem, int num_sms, int n_items, int ctas_per_sm = 0) {
    Schedule s;
    s.threads = NT;
    s.smem = smem;
    s.blocks = 0;  // 0: the largest work item does not fit one CTA
    int dev = 0, opt_in = 0;
    TFMM_CUDA_CHECK(cudaGetDevice(&dev));
    TFMM_CUDA_CHECK(cudaDeviceGetAttribute(&opt_in, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)opt_in) return s;
    if (smem > 48 * 1024)
        TFMM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TFMM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem));
    if (per_sm < 1) return s;
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    s.blocks = std::max(1, std::min(per_sm * num_sms, n_items));
    return s;
}

}  // namespace

Plan::~Plan() {
    auto F = [](void* p) { if (p) cudaFree(p); };
    F(d_grp_rwg); F(d_weights); F(d_counters); F(d_factors); F(d_items); F(d_agg_order); F(d_dis_order);
    F(d_dense); F(d_dense_items); F(d_dense_agg_order); F(d_dense_dis_order); F(d_geom);
    F(d_ws_x); F(d_ws_spec); F(d_ws_y);
    for (auto* a : f64_arenas) F(a);
}

void pack_factors_fp32(Plan& P, cudaStream_t s) {
    const int nt = P.n_theta, np = P.n_phi;
    P.items.assign((size_t)P.G * 2, TuckerItem{});
    int64_t off = 0, alg = 0;
    auto take = [&](int64_t elems) {
        const int64_t o = off;
        off += round_up(elems, 32);  // 256-byte aligned arrays
        return o;
    };
    P.max_nb = 0; P.max_ldnb = 0; P.max_ldab = 0;
    P.max_rank[0] = P.max_rank[1] = P.max_rank[2] = 0;
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            const int* rk = &P.ranks[((size_t)g * 2 + al) * 3];
            TuckerItem& d = P.items[(size_t)g * 2 + al];
            d.g = g;
            d.alpha = al;
            d.n_beta = (int)(P.grp_off[g + 1] - P.grp_off[g]);
            d.rwg = P.grp_off[g];
            d.rt = rk[0]; d.rp = rk[1]; d.rb = rk[2];
            d.ld_nb = (int)round_up(d.n_beta, 2);
            d.ld_ab = (int)round_up((int64_t)d.rt * d.rp, 2);
            d.ub = take((int64_t)d.rb * d.ld_nb);
            d.core = take((int64_t)d.rb * d.ld_ab);
            d.uphi = take((int64_t)np * d.rp);
            d.uth = take((int64_t)nt * d.rt);
            alg += (int64_t)d.rb * d.n_beta + (int64_t)d.rb * d.rt * d.rp;
            if (!plan_is_svd(P)) alg += (int64_t)np * d.rp + (int64_t)nt * d.rt;
            P.max_nb = std::max(P.max_nb, d.n_beta);
            P.max_ldnb = std::max(P.max_ldnb, d.ld_nb);
            P.max_ldab = std::max(P.max_ldab, d.ld_ab);
            P.max_rank[0] = std::max(P.max_rank[0], d.rt);
            P.max_rank[1] = std::max(P.max_rank[1], d.rp);
            P.max_rank[2] = std::max(P.max_rank[2], d.rb);
        }
    P.factor_elems = off;
    P.factor_elems_alg = alg;
    if (P.d_factors) cudaFree(P.d_factors);
    P.d_factors = nullptr;
    TFMM_CUDA_CHECK(device_malloc(&P.d_factors, sizeof(float2) * std::max<int64_t>(off, 1)));
    TFMM_CUDA_CHECK(cudaMemsetAsync(P.d_factors, 0, sizeof(float2) * std::max<int64_t>(off, 1), s));
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            const TuckerItem& d = P.items[(size_t)g * 2 + al];
            const HostFactors64& F = P.f64[(size_t)g * 2 + al];
            const double2* Ut = F.base;
            const double2* Up = Ut + (int64_t)nt * d.rt;
            const double2* Ub = Up + (int64_t)np * d.rp;
            const double2* Cc = Ub + (int64_t)d.n_beta * d.rb;
            const int m = d.rt * d.rp;
            to_f32_pad_kernel<<<grid1d((int64_t)d.n_beta * d.rb), 256, 0, s>>>(Ub, d.n_beta, d.rb, d.n_beta,
                                                                                P.d_factors + d.ub, d.ld_nb);
            to_f32_pad_kernel<<<grid1d((int64_t)m * d.rb), 256, 0, s>>>(Cc, m, d.rb, m, P.d_factors + d.core, d.ld_ab);
            to_f32_pad_kernel<<<grid1d((int64_t)np * d.rp), 256, 0, s>>>(Up, np, d.rp, np, P.d_factors + d.uphi, np);
            to_f32_pad_kernel<<<grid1d((int64_t)nt * d.rt), 256, 0, s>>>(Ut, nt, d.rt, nt, P.d_factors + d.uth, nt);
        }
    TFMM_CUDA_CHECK(cudaGetLastError());
    finalize_hot_layout(P, s);
}

void finalize_hot_layout(Plan& P, cudaStream_t s) {
    const int nI = P.G * 2;
    if (P.d_items) cudaFree(P.d_items);
    P.d_items = nullptr;
    TFMM_CUDA_CHECK(device_malloc(&P.d_items, sizeof(TuckerItem) * nI));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_items, P.items.data(), sizeof(TuckerItem) * nI, cudaMemcpyHostToDevice, s));
    configure_hot(P, P.tuning, s);
}

void configure_split(Plan& P, cudaStream_t s);

// Queue orders (0: most factor bytes first, the LPT rule; 1: group order) and
// persistent grids (threads per CTA, CTAs per SM capped by occupancy) of the
// two single-RHS kernels.
void configure_hot(Plan& P, const HotTuning& t, cudaStream_t s) {
    const int nI = P.G * 2;
    auto ok_threads = [](int nt) { return nt >= 64 && nt <= 512 && nt % 32 == 0; };
    TFMM_REQUIRE(ok_threads(t.agg_threads) && ok_threads(t.dis_threads), "threads per CTA must be 64..512, a multiple of 32");
    TFMM_REQUIRE(t.agg_ctas_per_sm >= 0 && t.dis_ctas_per_sm >= 0, "CTAs per SM must be >= 0");
    TFMM_REQUIRE((t.agg_order == 0 || t.agg_order == 1) && (t.dis_order == 0 || t.dis_order == 1), "order must be 0 or 1");
    TFMM_REQUIRE(t.split >= 0 && t.split <= 2, "split must be 0 (automatic), 1 (always) or 2 (never)");
    auto bytes = [&](const TuckerItem& d) {
        return (double)d.rb * d.ld_nb + (double)d.rb * d.ld_ab + (double)P.n_phi * d.rp + (double)P.n_theta * d.rt;
    };
    std::vector<int> agg(nI), dis(P.G);
    std::iota(agg.begin(), agg.end(), 0);
    std::iota(dis.begin(), dis.end(), 0);
    if (t.agg_order == 0)
        std::stable_sort(agg.begin(), agg.end(), [&](int a, int b) { return bytes(P.items[a]) > bytes(P.items[b]); });
    if (t.dis_order == 0)
        std::stable_sort(dis.begin(), dis.end(), [&](int a, int b) {
            return bytes(P.items[2 * a]) + bytes(P.items[2 * a + 1]) > bytes(P.items[2 * b]) + bytes(P.items[2 * b + 1]);
        });
    if (!P.d_agg_order) TFMM_CUDA_CHECK(device_malloc(&P.d_agg_order, sizeof(int) * nI));
    if (!P.d_dis_order) TFMM_CUDA_CHECK(device_malloc(&P.d_dis_order, sizeof(int) * std::max(P.G, 1)));
    // stream-ordered: launches already queued keep reading the old order until these copies land
    TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_agg_order, agg.data(), sizeof(int) * nI, cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_dis_order, dis.data(), sizeof(int) * P.G, cudaMemcpyHostToDevice, s));
    if (plan_is_svd(P)) {
        P.agg_sched = make_schedule(tucker_aggregate_kernel<true>, t.agg_threads,
                                    sizeof(float2) * svd_agg_layout(P, t.agg_threads).total, P.num_sms, nI,
                                    t.agg_ctas_per_sm);
        P.dis_sched = make_schedule(tucker_disaggregate_kernel<true>, t.dis_threads,
                                    sizeof(float2) * svd_dis_layout(P, t.dis_threads).total, P.num_sms, P.G,
                                    t.dis_ctas_per_sm);
    } else {
        P.agg_sched = make_schedule(tucker_aggregate_kernel<false>, t.agg_threads,
                                    sizeof(float2) * agg_layout(P, t.agg_threads).total, P.num_sms, nI,
                                    t.agg_ctas_per_sm);
        P.dis_sched = make_schedule(tucker_disaggregate_kernel<false>, t.dis_threads,
                                    sizeof(float2) * dis_layout(P, t.dis_threads).total, P.num_sms, P.G,
                                    t.dis_ctas_per_sm);
    }
    P.tuning = t;
    P.hot_ok = P.agg_sched.blocks > 0 && P.dis_sched.blocks > 0;
    const bool want_split = !plan_is_svd(P) && P.hot_ok && (t.split == 1 || (t.split == 0 && nI < 2 * P.num_sms));
    if (want_split != (bool)P.split) {  // captured graphs point into the split path's scratch
        TFMM_REQUIRE(P.live_graphs == 0, "destroy the plan's graphs before changing the single-RHS path");
        P.split.reset();
        if (want_split) configure_split(P, s);
    }
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
}

// Tile lists, scratch and shared-memory sizes of the split path.
void configure_split(Plan& P, cudaStream_t s) {
    auto SP = std::make_unique<SplitPlan>();
    const int nI = P.G * 2, NT = 512;
    std::vector<SplitTile> a1, a2, d2, d3;
    std::vector<int64_t> off(nI);
    int64_t tot = 0;
    for (int q = 0; q < nI; ++q) {
        const TuckerItem& d = P.items[q];
        off[q] = tot;
        tot += round_up(d.rb, 2) + d.ld_ab;
        for (int c = 0; c < d.rb; c += kSplitRows) {
            a1.push_back(SplitTile{q, c});
            d2.push_back(SplitTile{q, c});
        }
        for (int j = 0; j < d.ld_ab / 2; j += kSplitCols) a2.push_back(SplitTile{q, j});
    }
    for (int g = 0; g < P.G; ++g)
        for (int j = 0; j < P.items[2 * g].ld_nb / 2; j += kSplitCols) d3.push_back(SplitTile{g, j});
    auto up = [&](DeviceBuffer& b, const std::vector<SplitTile>& v, int& n) {
        n = (int)v.size();
        TFMM_CUDA_CHECK(device_malloc(&b.p, sizeof(SplitTile) * std::max<size_t>(v.size(), 1)));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(b.p, v.data(), sizeof(SplitTile) * v.size(), cudaMemcpyHostToDevice, s));
    };
    up(SP->t_ag1, a1, SP->n_ag1);
    up(SP->t_ag2, a2, SP->n_ag2);
    up(SP->t_dg2, d2, SP->n_dg2);
    up(SP->t_dg3, d3, SP->n_dg3);
    TFMM_CUDA_CHECK(device_malloc(&SP->scratch.p, sizeof(float2) * std::max<int64_t>(tot, 1)));
    TFMM_CUDA_CHECK(device_malloc(&SP->scr_off.p, sizeof(int64_t) * nI));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(SP->scr_off.p, off.data(), sizeof(int64_t) * nI, cudaMemcpyHostToDevice, s));
    SP->smem_ag1 = sizeof(float2) * al16(P.max_ldnb);
    SP->smem_ag2 = sizeof(float4) * NT + sizeof(float2) * al16(P.max_rank[2]);
    SP->smem_ag34 = sizeof(float2) * agg_layout(P, NT).total;
    SP->smem_dg1 = sizeof(float2) * dis_layout(P, NT).total;
    SP->smem_dg2 = sizeof(float2) * al16(P.max_ldab);
    SP->smem_dg3 = sizeof(float4) * (NT + kSplitCols) + sizeof(float2) * al16(P.max_rank[2]);
    auto allow = [](const void* k, size_t bytes) {
        if (bytes > 48 * 1024) TFMM_CUDA_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    };
    allow((const void*)split_ag1_kernel, SP->smem_ag1);
    allow((const void*)split_ag2_kernel, SP->smem_ag2);
    allow((const void*)split_ag34_kernel, SP->smem_ag34);
    allow((const void*)split_dg1_kernel, SP->smem_dg1);
    allow((const void*)split_dg2_kernel, SP->smem_dg2);
    allow((const void*)split_dg3_kernel, SP->smem_dg3);
    P.split = std::move(SP);
}

void finalize_dense_layout(Plan& P) {
    std::vector<DenseItem> items((size_t)P.G * 2);
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            DenseItem& d = items[(size_t)g * 2 + al];
            d.g = g;
            d.alpha = al;
            d.n_beta = (int)(P.grp_off[g + 1] - P.grp_off[g]);
            d.rwg = P.grp_off[g];
            d.a = ((int64_t)2 * P.grp_off[g] + (int64_t)al * d.n_beta) * P.ld_dir;
        }
    const int nI = P.G * 2;
    std::vector<int> agg(nI), dis(P.G);
    std::iota(agg.begin(), agg.end(), 0);
    std::iota(dis.begin(), dis.end(), 0);
    std::stable_sort(agg.begin(), agg.end(), [&](int a, int b) { return items[a].n_beta > items[b].n_beta; });
    std::stable_sort(dis.begin(), dis.end(), [&](int a, int b) { return items[2 * a].n_beta > items[2 * b].n_beta; });
    TFMM_CUDA_CHECK(device_malloc(&P.d_dense_items, sizeof(DenseItem) * nI));
    TFMM_CUDA_CHECK(cudaMemcpy(P.d_dense_items, items.data(), sizeof(DenseItem) * nI, cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(device_malloc(&P.d_dense_agg_order, sizeof(int) * nI));
    TFMM_CUDA_CHECK(device_malloc(&P.d_dense_dis_order, sizeof(int) * std::max(P.G, 1)));
    TFMM_CUDA_CHECK(cudaMemcpy(P.d_dense_agg_order, agg.data(), sizeof(int) * nI, cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(cudaMemcpy(P.d_dense_dis_order, dis.data(), sizeof(int) * P.G, cudaMemcpyHostToDevice));
    const int NT = 512;
    P.dagg_sched = make_schedule(dense_aggregate_kernel, NT, sizeof(float2) * (al16(P.max_nb) + 2 * NT), P.num_sms, nI);
    P.ddis_sched = make_schedule(dense_disaggregate_kernel, NT, sizeof(float2) * (P.ld_dir + al16(P.max_nb)),
                                 P.num_sms, P.G);
    TFMM_REQUIRE(P.dagg_sched.blocks > 0 && P.ddis_sched.blocks > 0,
                 "dense comparator: a group's RWGs or directions exceed one CTA's shared memory");
}

void pack_dense_fp32_from_f64(Plan& P, const double2* src, int g, int alpha, cudaStream_t s) {
    const int64_t nb = P.grp_off[g + 1] - P.grp_off[g];
    const int64_t dst = ((int64_t)2 * P.grp_off[g] + (int64_t)alpha * nb) * P.ld_dir;
    to_f32_pad_kernel<<<grid1d(P.n_dir * nb), 256, 0, s>>>(src, P.n_dir, nb, P.n_dir, P.d_dense + dst, P.ld_dir);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

namespace {

SplitArgs split_args(const Plan& P, int r) {
    SplitArgs a{};
    a.items = P.d_items;
    a.fac = P.d_factors;
    a.grp_rwg = P.d_grp_rwg;
    a.scratch = static_cast<float2*>(P.split->scratch.p);
    a.scr_off = static_cast<const int64_t*>(P.split->scr_off.p);
    a.n_theta = P.n_theta;
    a.n_phi = P.n_phi;
    a.n_dir = P.n_dir;
    a.G = P.G;
    a.r = r;
    return a;
}

void launch_split_aggregate(const Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    const SplitPlan& S = *P.split;
    for (int r = 0; r < R; ++r) {
        SplitArgs a = split_args(P, r);
        a.x = x;
        a.ldx = ldx;
        a.spec_out = spec;
        a.tiles = static_cast<const SplitTile*>(S.t_ag1.p);
        split_ag1_kernel<<<S.n_ag1, 512, S.smem_ag1, s>>>(a);
        a.tiles = static_cast<const SplitTile*>(S.t_ag2.p);
        split_ag2_kernel<<<S.n_ag2, 512, S.smem_ag2, s>>>(a);
        a.L = agg_layout(P, 512);
        split_ag34_kernel<<<P.G * 2, 512, S.smem_ag34, s>>>(a);
        TFMM_CUDA_CHECK(cudaGetLastError());
    }
}

void launch_split_disaggregate(const Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y,
                               int64_t ldy, cudaStream_t s) {
    const SplitPlan& S = *P.split;
    for (int r = 0; r < R; ++r) {
        SplitArgs a = split_args(P, r);
        a.spec = spec;
        a.w = weights ? P.d_weights : nullptr;
        a.y = y;
        a.ldy = ldy;
        a.beta = beta;
        a.L = dis_layout(P, 512);
        split_dg1_kernel<<<P.G * 2, 512, S.smem_dg1, s>>>(a);
        a.tiles = static_cast<const SplitTile*>(S.t_dg2.p);
        split_dg2_kernel<<<S.n_dg2, 512, S.smem_dg2, s>>>(a);
        a.tiles = static_cast<const SplitTile*>(S.t_dg3.p);
        split_dg3_kernel<<<S.n_dg3, 512, S.smem_dg3, s>>>(a);
        TFMM_CUDA_CHECK(cudaGetLastError());
    }
}

}  // namespace

void launch_tucker_aggregate(const Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    TFMM_REQUIRE(P.hot_ok, "single-RHS kernels unavailable for this plan (work item exceeds one CTA)");
    if (P.split) {
        launch_split_aggregate(P, x, R, ldx, spec, s);
        return;
    }
    AggArgs a;
    a.items = P.d_items;
    a.order = P.d_agg_order;
    a.n_items = P.G * 2;
    a.fac = P.d_factors;
    a.grp_rwg = P.d_grp_rwg;
    a.x = x;
    a.ldx = ldx;
    a.spec = spec;
    a.n_theta = P.n_theta;
    a.n_phi = P.n_phi;
    a.n_dir = P.n_dir;
    a.G = P.G;
    a.R = R;
    a.ctr = P.d_counters + 0;
    a.done = P.d_counters + 1;
    if (plan_is_svd(P)) {
        a.L = svd_agg_layout(P, P.agg_sched.threads);
        tucker_aggregate_kernel<true><<<P.agg_sched.blocks, P.agg_sched.threads, P.agg_sched.smem, s>>>(a);
    } else {
        a.L = agg_layout(P, P.agg_sched.threads);
        tucker_aggregate_kernel<false><<<P.agg_sched.blocks, P.agg_sched.threads, P.agg_sched.smem, s>>>(a);
    }
    TFMM_CUDA_CHECK(cudaGetLastError());
}

void launch_tucker_disaggregate(const Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y,
                                int64_t ldy, cudaStream_t s) {
    TFMM_REQUIRE(P.hot_ok, "single-RHS kernels unavailable for this plan (work item exceeds one CTA)");
    if (P.split) {
        launch_split_disaggregate(P, spec, R, weights, beta, y, ldy, s);
        return;
    }
    DisArgs a;
    a.items = P.d_items;
    a.order = P.d_dis_order;
    a.n_items = P.G;
    a.fac = P.d_factors;
    a.grp_rwg = P.d_grp_rwg;
    a.spec = spec;
    a.w = weights ? P.d_weights : nullptr;
    a.y = y;
    a.ldy = ldy;
    a.beta = beta;
    a.n_theta = P.n_theta;
    a.n_phi = P.n_phi;
    a.n_dir = P.n_dir;
    a.G = P.G;
    a.R = R;
    a.ctr = P.d_counters + 2;
    a.done = P.d_counters + 3;
    if (plan_is_svd(P)) {
        a.L = svd_dis_layout(P, P.dis_sched.threads);
        tucker_disaggregate_kernel<true><<<P.dis_sched.blocks, P.dis_sched.threads, P.dis_sched.smem, s>>>(a);
    } else {
        a.L = dis_layout(P, P.dis_sched.threads);
        tucker_disaggregate_kernel<false><<<P.dis_sched.blocks, P.dis_sched.threads, P.dis_sched.smem, s>>>(a);
    }
    TFMM_CUDA_CHECK(cudaGetLastError());
}

void launch_dense_aggregate(const Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    DenseAggArgs a;
    a.items = P.d_dense_items;
    a.order = P.d_dense_agg_order;
    a.n_items = P.G * 2;
    a.A = P.d_dense;
    a.grp_rwg = P.d_grp_rwg;
    a.x = x;
    a.ldx = ldx;
    a.spec = spec;
    a.n_dir = P.n_dir;
    a.ld_dir = P.ld_dir;
    a.G = P.G;
    a.R = R;
    a.part_off = al16(P.max_nb) / 2;
    a.ctr = P.d_counters + 4;
    a.done = P.d_counters + 5;
    dense_aggregate_kernel<<<P.dagg_sched.blocks, P.dagg_sched.threads, P.dagg_sched.smem, s>>>(a);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

void launch_dense_disaggregate(const Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y,
                               int64_t ldy, cudaStream_t s) {
    DenseDisArgs a;
    a.items = P.d_dense_items;
    a.order = P.d_dense_dis_order;
    a.n_items = P.G;
    a.A = P.d_dense;
    a.grp_rwg = P.d_grp_rwg;
    a.spec = spec;
    a.w = weights ? P.d_weights : nullptr;
    a.y = y;
    a.ldy = ldy;
    a.beta = beta;
    a.n_dir = P.n_dir;
    a.ld_dir = P.ld_dir;
    a.G = P.G;
    a.R = R;
    a.ctr = P.d_counters + 6;
    a.done = P.d_counters + 7;
    dense_disaggregate_kernel<<<P.ddis_sched.blocks, P.ddis_sched.threads, P.ddis_sched.smem, s>>>(a);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

}  // namespace tfmm
