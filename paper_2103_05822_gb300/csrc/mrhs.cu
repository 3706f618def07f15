// Multi-right-hand-side aggregation and disaggregation (Figs. 2b, 3b with R
// columns) as chains of grouped complex GEMMs, FP32 on CUDA cores.
//
// For R right-hand sides every step of the Tucker procedures becomes a small
// dense matrix product per (group, alpha).  Each step is one launch over all
// groups: a flat list of 64 x 64 output tiles, one CTA per tile.  Intermediates
// live in plan-owned scratch, in layouts chosen so that the next step reads
// them with plain strides:
//
//   aggregation, per (g, alpha):
//     AG1  T  (r_b x R)       = U_beta^T X_g           (X_g gathered from x)
//     AG2  M  (m x R)         = C_(3)^T T              m = r_t r_p, stored [b][r][a]
//     AG3  V  (n_phi x r_t R) = U_phi M'               stored [a][r][i_phi]
//     AG4  F  (n_theta x n_phi R) = U_theta V'         scattered into the spectra
//   disaggregation, per (g, alpha) then per g:
//     DG1a P  (r_t x n_phi R) = U_theta^T conj(W g)    stored [i_phi][r][a]
//     DG1b H  (r_t R x r_p)   = P' U_phi               stored [a + r_t b][r]
//     DG2  S  (r_b x R)       = C_(3) H
//     DG3  y_g = beta y_g + conj(U_beta^(0) S^(0) + U_beta^(1) S^(1))  (both alpha in one K loop)
#include <algorithm>
#include <vector>

#include "internal.h"

namespace tfmm {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NTH = 256;

enum Stage { AG1, AG2, AG3, AG4, DG1A, DG1B, DG2, DG3 };

struct Ctx {
    const float2* fac;   // packed FP32 factors
    const int* grp_rwg;  // RWG ids in group order
    const float2* in;    // stage input (x, spectra or the previous intermediate)
    float2* out;         // stage output (intermediate, spectra or y)
    const float* w;      // quadrature weights (DG1A) or null
    int64_t ld;          // ldx (AG1) / ldy (DG3)
    float2 beta;         // DG3
    int R, G, n_theta, n_phi, n_dir;
};

template <Stage S>
__device__ __forceinline__ float2 load_a(const Ctx& c, const MrProb& p, int i, int k) {
    switch (S) {
        case AG1: return c.fac[p.a0 + (int64_t)i * p.lda + k];                 // U_beta^T(c, n)
        case AG2: return c.fac[p.a0 + (int64_t)k * p.lda + i];                 // C_(3)^T(ab, c)
        case AG3: return c.fac[p.a0 + i + (int64_t)c.n_phi * k];               // U_phi(i_phi, b)
        case AG4: return c.fac[p.a0 + i + (int64_t)c.n_theta * k];             // U_theta(i_theta, a)
        case DG1A: return c.fac[p.a0 + k + (int64_t)c.n_theta * i];            // U_theta^T(a, i_theta)
        case DG1B: return c.in[p.b0 + i + (int64_t)p.rt * c.R * k];            // P'((a,r), i_phi)
        case DG2: return c.fac[p.a0 + (int64_t)i * p.lda + k];                 // C_(3)(c, ab)
        case DG3:                                                              // [U_b^(0) U_b^(1)](n, c)
            return k < p.K0 ? c.fac[p.a0 + (int64_t)k * p.lda + i] : c.fac[p.a1 + (int64_t)(k - p.K0) * p.lda + i];
    }
    return make_float2(0.f, 0.f);
}

template <Stage S>
__device__ __forceinline__ float2 load_b(const Ctx& c, const MrProb& p, int k, int j) {
    switch (S) {
        case AG1: return c.in[(int64_t)c.grp_rwg[p.rwg + k] + c.ld * j];       // x(n, r)
        case AG2: return c.in[p.b0 + k + (int64_t)p.rb * j];                   // T(c, r)
        case AG3: return c.in[p.b0 + (int64_t)k * p.rt * c.R + j];             // M'(b, (a, r))
        case AG4: return c.in[p.b0 + (int64_t)k * c.n_phi * c.R + j];          // V'(a, (i_phi, r))
        case DG1A: {                                                           // conj(W g)(i_theta, (i_phi, r))
            const int ip = j % c.n_phi, r = j / c.n_phi;
            const int o = k + c.n_theta * ip;
            const float2 v = c.in[(((int64_t)r * c.G + p.g) * 2 + p.alpha) * c.n_dir + o];
            const float wt = c.w ? c.w[o] : 1.0f;
            return make_float2(wt * v.x, -wt * v.y);
        }
        case DG1B: return c.fac[p.a0 + k + (int64_t)c.n_phi * j];              // U_phi(i_phi, b)
        case DG2: return c.in[p.b0 + k + (int64_t)p.m * j];                    // H(ab, r)
        case DG3:                                                              // [S^(0); S^(1)](c, r)
            return k < p.K0 ? c.in[p.b0 + k + (int64_t)p.K0 * j] : c.in[p.b1 + (k - p.K0) + (int64_t)(p.K - p.K0) * j];
    }
    return make_float2(0.f, 0.f);
}

template <Stage S>
__device__ __forceinline__ void store_c(const Ctx& c, const MrProb& p, int i, int j, float2 v) {
    switch (S) {
        case AG1: c.out[p.c0 + i + (int64_t)p.rb * j] = v; break;             // T(c, r)
        case AG2: {                                                            // M stored [b][r][a]
            const int a = i % p.rt, b = i / p.rt;
            c.out[p.c0 + a + (int64_t)p.rt * j + (int64_t)b * p.rt * c.R] = v;
        } break;
        case AG3: {                                                            // V stored [a][r][i_phi]
            const int a = j % p.rt, r = j / p.rt;
            c.out[p.c0 + (int64_t)a * c.n_phi * c.R + (int64_t)r * c.n_phi + i] = v;
        } break;
        case AG4: {                                                            // spectra
            const int ip = j % c.n_phi, r = j / c.n_phi;
            c.out[(((int64_t)r * c.G + p.g) * 2 + p.alpha) * c.n_dir + i + (int64_t)c.n_theta * ip] = v;
        } break;
        case DG1A: {                                                           // P stored [i_phi][r][a]
            const int ip = j % c.n_phi, r = j / c.n_phi;
            c.out[p.c0 + i + (int64_t)p.rt * r + (int64_t)p.rt * c.R * ip] = v;
        } break;
        case DG1B: {                                                           // H stored [a + r_t b][r]
            const int a = i % p.rt, r = i / p.rt;
            c.out[p.c0 + a + (int64_t)p.rt * j + (int64_t)p.m * r] = v;
        } break;
        case DG2: c.out[p.c0 + i + (int64_t)p.rb * j] = v; break;             // S(c, r)
        case DG3: {                                                            // y = beta y + conj(acc)
            float2* dst = c.out + (int64_t)c.grp_rwg[p.rwg + i] + c.ld * j;
            float2 r = make_float2(v.x, -v.y);
            if (c.beta.x != 0.f || c.beta.y != 0.f) {
                const float2 o = *dst;
                r.x += c.beta.x * o.x - c.beta.y * o.y;
                r.y += c.beta.x * o.y + c.beta.y * o.x;
            }
            *dst = r;
        } break;
    }
}

// One 64 x 64 complex output tile per CTA; 256 threads, 4 x 4 outputs each.
template <Stage S>
__global__ void __launch_bounds__(NTH) mr_gemm_kernel(const Ctx c, const MrProb* __restrict__ probs,
                                                      const MrTile* __restrict__ tiles) {
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN + 1];
    const MrTile t = tiles[blockIdx.x];
    const MrProb p = probs[t.prob];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    // consecutive threads walk the operand's contiguous index
    constexpr bool a_k = (S == AG1 || S == DG1A || S == DG2);
    constexpr bool b_k = !(S == AG3 || S == AG4);
    for (int k0 = 0; k0 < p.K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NTH) {
            const int ii = a_k ? e / BK : e % BM, kk = a_k ? e % BK : e / BM;
            const int i = t.m0 + ii, k = k0 + kk;
            As[kk][ii] = (i < p.M && k < p.K) ? load_a<S>(c, p, i, k) : make_float2(0.f, 0.f);
        }
        for (int e = tid; e < BN * BK; e += NTH) {
            const int jj = b_k ? e / BK : e % BN, kk = b_k ? e % BK : e / BN;
            const int j = t.n0 + jj, k = k0 + kk;
            Bs[kk][jj] = (j < p.N && k < p.K) ? load_b<S>(c, p, k, j) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            float2 av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fmaf(av[a].x, bv[b].x, acc[a][b].x);
                    acc[a][b].x = fmaf(-av[a].y, bv[b].y, acc[a][b].x);
                    acc[a][b].y = fmaf(av[a].x, bv[b].y, acc[a][b].y);
                    acc[a][b].y = fmaf(av[a].y, bv[b].x, acc[a][b].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = t.m0 + ty + 16 * a, j = t.n0 + tx + 16 * b;
            if (i < p.M && j < p.N) store_c<S>(c, p, i, j, acc[a][b]);
        }
}

void add_tiles(std::vector<MrTile>& tiles, int prob, int M, int N) {
    for (int m0 = 0; m0 < M; m0 += BM)
        for (int n0 = 0; n0 < N; n0 += BN) tiles.push_back(MrTile{prob, m0, n0});
}

template <Stage S>
void launch_stage(const Plan& P, const MrStage& st, Ctx c, cudaStream_t s) {
    if (st.n_tiles == 0) return;
    mr_gemm_kernel<S><<<st.n_tiles, NTH, 0, s>>>(c, st.d_probs, st.d_tiles);
    TFMM_CUDA_CHECK(cudaGetLastError());
    (void)P;
}

void upload_stage(MrStage& st, const std::vector<MrProb>& probs, const std::vector<MrTile>& tiles) {
    st.n_tiles = (int)tiles.size();
    TFMM_CUDA_CHECK(device_malloc(&st.d_probs, sizeof(MrProb) * std::max<size_t>(probs.size(), 1)));
    TFMM_CUDA_CHECK(device_malloc(&st.d_tiles, sizeof(MrTile) * std::max<size_t>(tiles.size(), 1)));
    TFMM_CUDA_CHECK(cudaMemcpy(st.d_probs, probs.data(), sizeof(MrProb) * probs.size(), cudaMemcpyHostToDevice));
    TFMM_CUDA_CHECK(cudaMemcpy(st.d_tiles, tiles.data(), sizeof(MrTile) * tiles.size(), cudaMemcpyHostToDevice));
}

}  // namespace

MrStage::~MrStage() {
    if (d_probs) cudaFree(d_probs);
    if (d_tiles) cudaFree(d_tiles);
}

MrPlan::~MrPlan() {
    if (buf[0]) cudaFree(buf[0]);
    if (buf[1]) cudaFree(buf[1]);
    if (buf[2]) cudaFree(buf[2]);
}

// Problem and tile lists of every stage for R right-hand sides, plus scratch.
MrPlan* get_mr_plan(Plan& P, int R) {
    for (auto& m : P.mr)
        if (m->R == R) return m.get();
    auto mp = std::make_unique<MrPlan>();
    MrPlan& M = *mp;
    M.R = R;
    const int nt = P.n_theta, np = P.n_phi;
    int64_t off1 = 0, off2 = 0, off3 = 0;  // scratch sizes: T/S, M/H, V/P
    std::vector<int64_t> o1(P.G * 2), o2(P.G * 2), o3(P.G * 2);
    for (int q = 0; q < P.G * 2; ++q) {
        const TuckerItem& d = P.items[q];
        const int m = d.rt * d.rp;
        o1[q] = off1;
        off1 += (int64_t)d.rb * R;
        o2[q] = off2;
        off2 += (int64_t)m * R;
        o3[q] = off3;
        off3 += (int64_t)std::max(np, nt) * d.rt * R;
    }
    TFMM_CUDA_CHECK(device_malloc(&M.buf[0], sizeof(float2) * std::max<int64_t>(off1, 1)));
    TFMM_CUDA_CHECK(device_malloc(&M.buf[1], sizeof(float2) * std::max<int64_t>(off2, 1)));
    TFMM_CUDA_CHECK(device_malloc(&M.buf[2], sizeof(float2) * std::max<int64_t>(off3, 1)));
    std::vector<MrProb> pr[8];
    std::vector<MrTile> tl[8];
    for (int q = 0; q < P.G * 2; ++q) {
        const TuckerItem& d = P.items[q];
        const int m = d.rt * d.rp;
        MrProb b{};
        b.g = d.g;
        b.alpha = d.alpha;
        b.rt = d.rt;
        b.rb = d.rb;
        b.m = m;
        b.rwg = d.rwg;
        // AG1: T = U_beta^T X_g
        MrProb p = b;
        p.M = d.rb; p.N = R; p.K = d.n_beta; p.a0 = d.ub; p.lda = d.ld_nb; p.c0 = o1[q];
        add_tiles(tl[AG1], (int)pr[AG1].size(), p.M, p.N); pr[AG1].push_back(p);
        // AG2: M = C_(3)^T T
        p = b;
        p.M = m; p.N = R; p.K = d.rb; p.a0 = d.core; p.lda = d.ld_ab; p.b0 = o1[q]; p.c0 = o2[q];
        add_tiles(tl[AG2], (int)pr[AG2].size(), p.M, p.N); pr[AG2].push_back(p);
        // AG3: V = U_phi M'
        p = b;
        p.M = np; p.N = d.rt * R; p.K = d.rp; p.a0 = d.uphi; p.b0 = o2[q]; p.c0 = o3[q];
        add_tiles(tl[AG3], (int)pr[AG3].size(), p.M, p.N); pr[AG3].push_back(p);
        // AG4: F = U_theta V'
        p = b;
        p.M = nt; p.N = np * R; p.K = d.rt; p.a0 = d.uth; p.b0 = o3[q];
        add_tiles(tl[AG4], (int)pr[AG4].size(), p.M, p.N); pr[AG4].push_back(p);
        // DG1a: P = U_theta^T conj(W g)
        p = b;
        p.M = d.rt; p.N = np * R; p.K = nt; p.a0 = d.uth; p.c0 = o3[q];
        add_tiles(tl[DG1A], (int)pr[DG1A].size(), p.M, p.N); pr[DG1A].push_back(p);
        // DG1b: H = P' U_phi
        p = b;
        p.M = d.rt * R; p.N = d.rp; p.K = np; p.a0 = d.uphi; p.b0 = o3[q]; p.c0 = o2[q];
        add_tiles(tl[DG1B], (int)pr[DG1B].size(), p.M, p.N); pr[DG1B].push_back(p);
        // DG2: S = C_(3) H
        p = b;
        p.M = d.rb; p.N = R; p.K = m; p.a0 = d.core; p.lda = d.ld_ab; p.b0 = o2[q]; p.c0 = o1[q];
        add_tiles(tl[DG2], (int)pr[DG2].size(), p.M, p.N); pr[DG2].push_back(p);
    }
    for (int g = 0; g < P.G; ++g) {
        const TuckerItem& d0 = P.items[2 * g];
        const TuckerItem& d1 = P.items[2 * g + 1];
        MrProb p{};
        p.g = g;
        p.M = d0.n_beta; p.N = R; p.K0 = d0.rb; p.K = d0.rb + d1.rb;
        p.a0 = d0.ub; p.a1 = d1.ub; p.lda = d0.ld_nb;
        p.b0 = o1[2 * g]; p.b1 = o1[2 * g + 1];
        p.rwg = d0.rwg;
        add_tiles(tl[DG3], (int)pr[DG3].size(), p.M, p.N); pr[DG3].push_back(p);
    }
    for (int s = 0; s < 8; ++s) upload_stage(M.st[s], pr[s], tl[s]);
    P.mr.push_back(std::move(mp));
    return P.mr.back().get();
}

void launch_mr_aggregate(Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    MrPlan* M = get_mr_plan(P, R);
    Ctx c{};
    c.fac = P.d_factors;
    c.grp_rwg = P.d_grp_rwg;
    c.R = R; c.G = P.G; c.n_theta = P.n_theta; c.n_phi = P.n_phi; c.n_dir = P.n_dir;
    c.ld = ldx;
    c.in = x; c.out = M->buf[0];
    launch_stage<AG1>(P, M->st[AG1], c, s);
    c.in = M->buf[0]; c.out = M->buf[1];
    launch_stage<AG2>(P, M->st[AG2], c, s);
    c.in = M->buf[1]; c.out = M->buf[2];
    launch_stage<AG3>(P, M->st[AG3], c, s);
    c.in = M->buf[2]; c.out = spec;
    launch_stage<AG4>(P, M->st[AG4], c, s);
}

void launch_mr_disaggregate(Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y, int64_t ldy,
                            cudaStream_t s) {
    MrPlan* M = get_mr_plan(P, R);
    Ctx c{};
    c.fac = P.d_factors;
    c.grp_rwg = P.d_grp_rwg;
    c.R = R; c.G = P.G; c.n_theta = P.n_theta; c.n_phi = P.n_phi; c.n_dir = P.n_dir;
    c.w = weights ? P.d_weights : nullptr;
    c.in = spec; c.out = M->buf[2];
    launch_stage<DG1A>(P, M->st[DG1A], c, s);
    c.in = M->buf[2]; c.out = M->buf[1];
    launch_stage<DG1B>(P, M->st[DG1B], c, s);
    c.in = M->buf[1]; c.out = M->buf[0];
    launch_stage<DG2>(P, M->st[DG2], c, s);
    c.in = M->buf[0]; c.out = y; c.ld = ldy; c.beta = beta;
    launch_stage<DG3>(P, M->st[DG3], c, s);
}

}  // namespace tfmm
