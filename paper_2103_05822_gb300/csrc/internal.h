// Internal declarations shared by the tfmm translation units (not installed).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tfmm.h"

namespace tfmm {

struct Error : std::runtime_error {
    tfmm_status code;
    Error(tfmm_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(tfmm_status c, const std::string& m) { throw Error(c, m); }

#define TFMM_CUDA_CHECK(call)                                                                       \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            if (e_ == cudaErrorMemoryAllocation)                                                    \
                ::tfmm::fail(TFMM_OOM, std::string(#call) + ": " + cudaGetErrorString(e_));         \
            ::tfmm::fail(TFMM_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
        }                                                                                           \
    } while (0)

// Every device allocation of the library goes through device_malloc, so that the
// test hook tfmm_test_fail_allocation can make the n-th one fail (TFMM_OOM).
cudaError_t device_malloc_bytes(void** p, size_t bytes);
template <class T>
inline cudaError_t device_malloc(T** p, size_t bytes) {
    return device_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}

#define TFMM_REQUIRE(cond, msg)                                                                     \
    do {                                                                                            \
        if (!(cond)) ::tfmm::fail(TFMM_INVALID_ARG, msg);                                           \
    } while (0)

// ----------------------------------------------------------------------- mesh
struct Mesh {
    int64_t nv = 0, nt = 0;
    std::vector<double> verts;   // nv x 3
    std::vector<int32_t> tris;   // nt x 3
    int64_t n_rwg = 0;
    std::vector<int64_t> edge;   // n_rwg x 2, ascending vertex ids
    std::vector<int64_t> tri;    // n_rwg x 2, (T+, T-)
    std::vector<int64_t> freev;  // n_rwg x 2, (p+, p-)
    std::vector<double> length;  // n_rwg
};

// RWG geometry as the far-field kernels read it: p+, p-, q1, q2 (edge ends), l.
struct RwgGeom {
    double pp[3], pm[3], q1[3], q2[3];
    double l, pad[3];
};

// ---------------------------------------------------------------- hot layout
// One (group, alpha) work item of the Tucker kernels.  Offsets count complex
// elements in the packed FP32 factor buffer; every array starts 16-byte aligned.
struct TuckerItem {
    int64_t ub;    // U_beta^T: r_b rows of ld_nb (row c = column c of U_beta)
    int64_t core;  // C_(3): r_b rows of ld_ab, entry a + r_t b
    int64_t uphi;  // U_phi, n_phi x r_p column-major
    int64_t uth;   // U_theta, n_theta x r_t column-major
    int64_t rwg;   // offset of the group's RWG ids
    int32_t n_beta, ld_nb, rt, rp, rb, ld_ab, g, alpha;
};

// One (group, alpha) uncompressed tensor: n_beta rows of ld_dir (row n = P_n^{alpha,+}).
struct DenseItem {
    int64_t a;
    int64_t rwg;
    int32_t n_beta, g, alpha, pad;
};

// Multi-RHS GEMM chain: one small complex GEMM per (group, alpha) and stage.
struct MrProb {
    int M, N, K, K0;       // K0: length of the first K segment (disaggregation's last stage)
    int g, alpha, rt, rb, m, lda;
    int64_t a0, a1;        // factor offsets (a1: second K segment)
    int64_t b0, b1;        // input offsets (b1: second K segment)
    int64_t c0;            // output offset
    int64_t rwg;           // offset of the group's RWG ids
};
struct MrTile {
    int prob, m0, n0;
};
struct MrStage {
    MrProb* d_probs = nullptr;
    MrTile* d_tiles = nullptr;
    int n_tiles = 0;
    ~MrStage();
};
struct MrPlan {             // per R: problem / tile lists of the 8 stages and scratch
    int R = 0;
    MrStage st[8];
    float2* buf[3] = {nullptr, nullptr, nullptr};
    ~MrPlan();
};

// Tensor-core (split-BF16) multi-RHS chain.
// Owns one device allocation (freed with its owner).
struct DeviceBuffer {
    void* p = nullptr;
    DeviceBuffer() = default;
    DeviceBuffer(const DeviceBuffer&) = delete;
    DeviceBuffer& operator=(const DeviceBuffer&) = delete;
    ~DeviceBuffer() {
        if (p) cudaFree(p);
    }
};

struct TcMat {              // 2T bfloat16 planes of one matrix, rows x ld (K-major, zero padded)
    int64_t off = 0;
    int64_t ld = 0;
    int rows = 0;
};
struct TcItem {             // the two K-major layouts of every factor of one (group, alpha)
    TcMat ubT, ub, c3T, c3, uphT, uph, uthT, uth;
};
struct TcProb {             // one grouped-GEMM problem D (M x N) = A (M x K) B (K x N), complex
    int M, N, K0, K1, BN;   // K1 > 0: a second K segment (A1, B1)
    const __nv_bfloat16* A0; int64_t a_ld0, a_ps0;
    const __nv_bfloat16* B0; int64_t b_ld0, b_ps0;
    const __nv_bfloat16* A1; int64_t a_ld1, a_ps1;
    const __nv_bfloat16* B1; int64_t b_ld1, b_ps1;
    void* out; int64_t o_ld, o_ps;
    int g, alpha, rt, n_phi;
    int64_t rwg;
};
struct TcStagePlan {
    TcProb* d_probs = nullptr;
    MrTile* d_tiles = nullptr;
    void* d_maps = nullptr;       // CUtensorMap x 4 per problem (A0, B0, A1, B1) when TMA feeds the stage
    int n_tiles = 0, n_probs = 0;
    int max_kt = 1, max_bn = 16;  // largest K-tile count and BN over the stage's problems
    ~TcStagePlan();
};
// Fused AG3 + AG4 (one launch): padded operand sizes shared by all its CTAs.
struct FusedShape {
    int K1 = 0, K2 = 0;      // r_phi and r_theta padded to 16 (the two contraction depths)
    int N1p = 0, N1s = 0;    // largest r_theta x (RHS per CTA), padded to 16 (MMA N) and 32 (TMEM spacing)
    int ntp = 0, nt32 = 0;   // n_theta padded to 16 (MMA N) and 32 (TMEM spacing)
    int nbuf = 2;            // AG4 accumulator sets in flight (1 or 2)
    int nacc = 1;            // accumulators per set (1 or 2), each 2 ntp columns [re | im]
    int tcols = 0;           // TMEM columns per CTA
    size_t smem = 0;         // dynamic shared memory per CTA
};

// DG1a or DG1b with the BF16 terms of the factor stacked along N (tc_cat_kernel)
struct CatPlan {
    bool on = false;
    int K = 0, K16 = 0, n8max = 0, tcols = 0, ntiles = 0;
    size_t smem = 0;
    DeviceBuffer items, tiles;
};

struct TcPlan {             // per (R, terms): problem lists of the 8 steps and scratch planes
    int R = 0, T = 0;
    TcStagePlan st[8];
    void* buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // fused AG3 + AG4, when every item fits one CTA (else the two stages run apart)
    bool fused34 = false;
    FusedShape f34;
    DeviceBuffer f34_items, f34_tiles;
    int f34_ntiles = 0;
    // DG1a with (i_phi, r) pairs as the MMA N dimension
    bool dg1a = false;
    int dg1a_K = 0, dg1a_NP = 0, dg1a_AR = 0, dg1a_ntiles = 0;
    size_t dg1a_smem = 0;
    DeviceBuffer dg1a_items, dg1a_tiles;
    CatPlan cat1a, cat1b;   // the stacked-term forms of DG1a / DG1b, when they fit
    // per item: element offsets of its M' and V'' / P'' scratch planes (for re-planning)
    std::vector<int64_t> m_off, v_off;
    ~TcPlan();
};

// Translation stage (FMM-FFT): zero-padded box grid, transform of the translation
// kernel and the cuFFT plan of the hot path (built on first use).
struct TransPlan {
    int N[3] = {1, 1, 1};    // FFT grid N_x, N_y, N_z >= 2K - 1
    int64_t Ns = 0;          // grid points
    int nb = 0;              // interleaved transforms per right-hand side: 2 N_dir
    int fft = 0;             // cufftHandle (C2C, nb transforms)
    DeviceBuffer That;       // N_dir x Ns FP32 complex: transform of (-jk/16 pi^2) T_L over the grid
    DeviceBuffer grid;       // nb x Ns FP32 complex work array (one transform after the other)
    DeviceBuffer group_cell; // G int: grid point of each group
    ~TransPlan();
};

// Launch shape and queue order of the single-RHS kernels (set by the autotuner).
struct HotTuning {
    int agg_threads = 512, agg_ctas_per_sm = 0, agg_order = 0;  // ctas 0: as many as fit
    int dis_threads = 512, dis_ctas_per_sm = 0, dis_order = 0;  // order 0: longest first, 1: group order
    int split = 0;  // split path: 0 automatic (fewer work items than 2 x SMs), 1 always, 2 never
};

// Split path of the single-RHS stages (plans with few, large items): tile lists of the
// row- and column-block launches and the items' intermediates.
struct SplitPlan {
    DeviceBuffer t_ag1, t_ag2, t_dg2, t_dg3;  // SplitTile lists
    int n_ag1 = 0, n_ag2 = 0, n_dg2 = 0, n_dg3 = 0;
    DeviceBuffer scratch;                     // per item: r_beta (padded to 2) + ld_ab complex
    DeviceBuffer scr_off;                     // per item: offset of its slot (complex elements)
    size_t smem_ag1 = 0, smem_ag2 = 0, smem_ag34 = 0, smem_dg1 = 0, smem_dg2 = 0, smem_dg3 = 0;
};

struct Schedule {
    int threads = 512;
    int blocks = 0;       // persistent grid
    size_t smem = 0;      // dynamic shared memory per CTA
};

// ----------------------------------------------------------------------- plan
struct HostFactors64 {     // FP64 factors of one (g, alpha), device memory (inside an arena)
    double2* base = nullptr;  // U_theta | U_phi | U_beta | core (column-major, back to back)
    int rt = 0, rp = 0, rb = 0;
};

struct Plan {
    // grid
    int L = 0, n_theta = 0, n_phi = 0, n_dir = 0, ld_dir = 0;
    std::vector<double> theta, w_theta, phi;
    double w_phi = 0.0;
    std::vector<float> weights;         // n_dir
    double k = 0.0;
    // groups
    int G = 0;
    int64_t N = 0;
    int K[3] = {1, 1, 1};
    std::vector<int64_t> grp_off;      // G + 1
    std::vector<int64_t> grp_rwg;      // N
    std::vector<double> centres;       // G x 3
    std::vector<int32_t> ranks;        // G x 2 x 3
    bool has_geometry = false;
    tfmm_params params{};
    double setup_ms[4] = {0, 0, 0, 0};

    // device: common
    int* d_grp_rwg = nullptr;          // N (int32 global RWG ids, group order)
    float* d_weights = nullptr;        // n_dir
    unsigned int* d_counters = nullptr;// work-queue tickets (self-resetting)
    int num_sms = 0;
    // device: Tucker
    float2* d_factors = nullptr;
    int64_t factor_elems = 0, factor_elems_alg = 0;
    TuckerItem* d_items = nullptr;     // G x 2, (g, alpha) order
    int* d_agg_order = nullptr;        // item ids, longest first
    int* d_dis_order = nullptr;        // group ids, longest first
    std::vector<TuckerItem> items;
    Schedule agg_sched, dis_sched;
    HotTuning tuning;
    int tc_f34_n1 = 0;                 // cap on r_theta x RHS per CTA of the fused AG3+AG4 kernel (0: largest that fits)
    int tc_dg1a_pairs = 0;             // (i_phi, r) pairs per CTA of the DG1a kernel (0: 128 when it fits, else 64)
    bool hot_ok = false;               // the single-RHS kernels fit (shared memory of the largest item)
    std::unique_ptr<SplitPlan> split;  // set when the single-RHS stages run the split path
    double tuned_ms[2] = {0, 0};       // autotuner's best aggregate / disaggregate times
    int live_graphs = 0;               // captured graphs that still point into this plan
    int max_nb = 0, max_ldnb = 0, max_rank[3] = {0, 0, 0}, max_ldab = 0;
    // device: dense
    float2* d_dense = nullptr;
    int64_t dense_elems = 0;
    DenseItem* d_dense_items = nullptr;
    int* d_dense_agg_order = nullptr;
    int* d_dense_dis_order = nullptr;
    Schedule dagg_sched, ddis_sched;
    // device: geometry for recomputation / excitation
    RwgGeom* d_geom = nullptr;         // N, global RWG order
    std::vector<RwgGeom> geom;
    // FP64 factors (exports)
    std::vector<HostFactors64> f64;    // G x 2, pointers into f64_arenas
    std::vector<double2*> f64_arenas;  // owned device allocations
    // multi-RHS chains, one per R used so far
    std::vector<std::unique_ptr<MrPlan>> mr;
    // tensor-core chains: factor planes (built on first use) and one chain per (R, terms)
    DeviceBuffer tc_fac[4];            // [T]: bf16 planes of every factor, T = 2, 3 (kept: chains point here)
    std::vector<TcItem> tc_items[4];
    DeviceBuffer tc_err;               // int: waits that gave up
    std::vector<std::unique_ptr<TcPlan>> tc;
    // translation stage (built on the first tfmm_translate)
    std::unique_ptr<TransPlan> trans;
    // workspace of tfmm_matvec_host
    int ws_R = 0;
    float2 *d_ws_x = nullptr, *d_ws_spec = nullptr, *d_ws_y = nullptr;

    ~Plan();
};

// tfmm_host.cpp
std::string& last_error();  // message of the calling thread's last failure
void upload_common(Plan& P, cudaStream_t s);

template <class F>
tfmm_status guarded(F&& f) {
    try {
        last_error().clear();
        f();
        return TFMM_OK;
    } catch (const Error& e) {
        last_error() = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        last_error() = "host allocation failed";
        return TFMM_OOM;
    } catch (const std::exception& e) {
        last_error() = e.what();
        return TFMM_INVALID_ARG;
    }
}

// setup.cu
void build_tucker_setup(Plan& P, const Mesh& M, cudaStream_t s);
void farfield_group_host(const Plan& P, int g, double2* At, double2* Ap, cudaStream_t s);
void planewave_rhs(const Plan& P, const double* khat, const double* pol, int R, float2* V, cudaStream_t s);
void planewave_rhs_noalloc(const Plan& P, const double* khat, const double* pol, int R, float2* V, cudaStream_t s);
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// apply.cu
void finalize_hot_layout(Plan& P, cudaStream_t s);  // items, schedules, orders (factors already packed)
void finalize_dense_layout(Plan& P);
void launch_tucker_aggregate(const Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s);
void launch_tucker_disaggregate(const Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y,
                                int64_t ldy, cudaStream_t s);
void launch_dense_aggregate(const Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s);
void launch_dense_disaggregate(const Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y,
                               int64_t ldy, cudaStream_t s);
void pack_factors_fp32(Plan& P, cudaStream_t s);  // from P.f64 into P.d_factors
void configure_hot(Plan& P, const HotTuning& t, cudaStream_t s);  // orders and schedules of the 1-RHS kernels
// mrhs_tc.cu
void build_tc_factors(Plan& P, int T, cudaStream_t s);
TcPlan* get_tc_plan(Plan& P, int R, int T, cudaStream_t s);
void tc_replan_shapes(Plan& P);  // re-plans the fused AG3+AG4 and DG1a kernels of every chain after a preference change
void launch_tc_aggregate(Plan& P, int T, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s);
void launch_tc_disaggregate(Plan& P, int T, const float2* spec, int R, int weights, float2 beta, float2* y,
                            int64_t ldy, cudaStream_t s);
// translate.cu
void build_translation(Plan& P, cudaStream_t s);
void launch_translate(Plan& P, const float2* spec_out, int R, float2* spec_in, cudaStream_t s);
// mrhs.cu
MrPlan* get_mr_plan(Plan& P, int R);
void launch_mr_aggregate(Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s);
void launch_mr_disaggregate(Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y, int64_t ldy,
                            cudaStream_t s);
void pack_dense_fp32_from_f64(Plan& P, const double2* src, int g, int alpha, cudaStream_t s);

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// The plan holds the truncated SVD of the aggregation matrices (identity theta / phi factors).
inline bool plan_is_svd(const Plan& P) { return P.params.compression == 1; }

}  // namespace tfmm

struct tfmm_mesh {
    tfmm::Mesh m;
};
struct tfmm_plan {
    tfmm::Plan p;
};
