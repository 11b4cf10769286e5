// rbe_api.cu -- host side of the C ABI declared in include/rbe.h.
//
// Builds, in FP64 on the host, everything that is fixed per system: the
// per-axis inverse-CDF table of the k distribution (Eq. probexpression with the
// per-axis marginal exp(-pi^2 m^2 / (alpha L^2))), H (Eq. psf) and S = H^3 - 1
// (Eq. S), the coefficient scales of Eq. rbmapprox and of the energy, the LJ
// shift of Eq. Ljpotential and the Langevin constants of Sec. 3.3.  Then it
// enqueues the kernels of one evaluation / MD step on the handle's stream.
//
// Sampling table (the exact arithmetic both this library and any independent
// implementation must follow to draw the same k):
//   M   = ceil( sqrt(alpha L^2 * 64 ln 2) / pi )
//   a   = pi^2 / (alpha L^2);  w_j = exp(-(a * (j - M)^2)),  j = 0 .. 2M
//   Z   = sum_j w_j in increasing j;   c_j = running sum in increasing j
//   T_j = min(floor((c_j / Z) * 2^32), 2^32 - 1) for j < 2M;  T_2M = 2^32
//   H   = Z,  S = H^3 - 1.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "rbe.h"
#include "rbe_internal.cuh"

using namespace rbe;

namespace {

thread_local std::string g_last_error;

struct SysHost {
    rbe_params p;
    int n = 0;
    int M = 0;
    double H = 0.0, S = 0.0;
    int ncd = 0;
    double skin = 0.0;                 // neighbour-list skin in effect (0 without a list)
    std::vector<uint64_t> table;
    std::vector<uint64_t> mh_tq;       // MH proposal thresholds (2M+1)
    std::vector<double> mh_rho;        // MH target / proposal ratios (2M+1)
    int off_p = 0, off_c = 0, off_k = 0, off_t = 0;
};

struct GraphEntry {
    int n;
    const void* pos;
    const void* vel;
    const void* step;
    const void* F;
    int prec;
    const void* host_pos;  // host-buffer graphs: the caller's pinned arrays (else null)
    const void* host_vel;
    int host_steps;        // host-buffer graphs: steps per replay
    const void* done;      // completion word of a zero-copy host step (else null)
    cudaGraphExec_t exec;
    int kernels;           // kernels in one replay
};

int axis_M(double alpha, double L) {
    const double x = std::sqrt(alpha * L * L * (64.0 * std::log(2.0))) / M_PI;
    return (int)std::ceil(x);
}

double build_table(double alpha, double L, int M, std::vector<uint64_t>& T) {
    const double a = (M_PI * M_PI) / (alpha * L * L);
    const int n = 2 * M + 1;
    T.assign(n, 0);
    double Z = 0.0;
    for (int j = 0; j < n; ++j) {
        const long long d = (long long)(j - M);
        Z += std::exp(-(a * (double)(d * d)));
    }
    double cum = 0.0;
    for (int j = 0; j < n; ++j) {
        const long long d = (long long)(j - M);
        cum += std::exp(-(a * (double)(d * d)));
        if (j == n - 1) {
            T[j] = 4294967296ull;
        } else {
            double f = std::floor((cum / Z) * 4294967296.0);
            if (f > 4294967295.0) f = 4294967295.0;
            T[j] = (uint64_t)f;
        }
    }
    return Z;
}

// Tables of the paper's Metropolis-Hastings sampler (Sec. 3.1) over |m| <= M,
// index j = m + M.  The proposal m* = round(x*), x* ~ N(0, alpha L^2 / (2 pi^2)),
// has the pmf qbar(0) = erf(1/(2s)), qbar(m) = (erf((|m|+1/2)/s) - erf((|m|-1/2)/s))/2
// with s = sqrt(alpha) L / pi, evaluated through erfc so the tails keep their
// precision.  tq[j] = floor(2^32 CDF_qbar(j)) (tq[2M] = 2^32) draws m* from a
// 32-bit word; rho[j] = exp(-pi^2 m^2 / (alpha L^2)) / qbar(m) gives the
// acceptance test u * rho(m) < rho(m*) of the independence sampler.
void build_mh_tables(double alpha, double L, int M, std::vector<uint64_t>& tq,
                     std::vector<double>& rho) {
    const int n = 2 * M + 1;
    const double s = std::sqrt(alpha) * L / M_PI;
    const double a = (M_PI * M_PI) / (alpha * L * L);
    std::vector<double> qb(n);
    double Q = 0.0;
    for (int j = 0; j < n; ++j) {
        const int m = std::abs(j - M);
        qb[j] = m == 0 ? std::erf(0.5 / s)
                       : 0.5 * (std::erfc(((double)m - 0.5) / s) - std::erfc(((double)m + 0.5) / s));
        Q += qb[j];
    }
    tq.assign(n, 0);
    rho.assign(n, 0.0);
    double cum = 0.0;
    for (int j = 0; j < n; ++j) {
        cum += qb[j];
        if (j == n - 1) {
            tq[j] = 4294967296ull;
        } else {
            double f = std::floor((cum / Q) * 4294967296.0);
            if (f > 4294967295.0) f = 4294967295.0;
            tq[j] = (uint64_t)f;
        }
        const long long d = (long long)(j - M);
        rho[j] = std::exp(-(a * (double)(d * d))) / qb[j];
    }
}

int pow2_ceil(long long v) {
    int p = 1;
    while (p < v && p < (1 << 30)) p <<= 1;
    return p;
}

template <class T>
rbe_status dalloc(T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc((void**)ptr, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return RBE_ERR_OOM;
    }
    return RBE_OK;
}

}  // namespace

struct rbe_ctx {
    bool batch = false;
    int nsys = 0;
    int ntot = 0;          // particle capacity (batch: exact total)
    int ncell = 0;
    int ktot = 0;
    int ttot = 0;
    int pmax = 0;
    std::vector<SysHost> sys;
    std::vector<SysDev> sysdev;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t stream2 = nullptr;          // Fourier branch of each evaluation
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int rho_chunk = 0, force_split = 0, real_split = 0, real_seg = 0;   // 0 = automatic
    int cur_n = -1, cur_chunk = -1, cur_split = -1, cur_rsplit = -1, cur_seg = -1;
    int npblk = 0, nfblk = 0, nrblk = 0, nchunks = 0, split = 1, rsplit = 1;
    int nseg = 0, seg_max = 1, stage_cap = 0, seg_threads = 64;
    int max_pblk = 0, max_fblk = 0, max_rblk = 0, max_chunks = 0, max_seg = 0;
    size_t max_part = 0;
    bool use_graph = false;
    double wait_limit = 0.0;                  // seconds a host wait may take (0: no limit)
    // list steps: structure factors + standing-list pass in one launch:
    // fusion_mode -1 automatic, 0 off, 1 on; fuse_tuned the autotuner's choice
    // (-1 before the first autotune: then systems of kFuseMinN particles and
    // more fuse)
    int fusion_mode = -1;
    int fuse_tuned = -1;
    std::vector<GraphEntry> graphs;
    std::string err;
    // per-kernel profile
    bool prof_on = false;
    cudaEvent_t ev_beg[RBE_K_COUNT] = {};
    cudaEvent_t ev_end[RBE_K_COUNT] = {};
    double prof_ms[RBE_K_COUNT] = {};
    int64_t prof_cnt[RBE_K_COUNT] = {};
    int64_t kernel_count = 0;

    SysDev* d_sys = nullptr;
    Tile* d_pblk = nullptr;
    Tile* d_fblk = nullptr;
    Tile* d_rblk = nullptr;
    Tile* d_segs = nullptr;
    Tile* d_chunks = nullptr;
    int* d_kstart = nullptr;
    int* d_cstart = nullptr;
    uint64_t* d_table = nullptr;
    uint4* d_fx = nullptr;
    uint4* d_spos = nullptr;
    double4* d_fx64 = nullptr;
    double4* d_spos64 = nullptr;
    int* d_cid = nullptr;
    int* d_rank = nullptr;
    int* d_perm = nullptr;
    int* d_perm_tmp = nullptr;
    float4* d_fs = nullptr;
    double4* d_fs64 = nullptr;
    int* d_cell_cnt = nullptr;
    int* d_cell_start = nullptr;
    int4* d_ksamp = nullptr;
    unsigned long long* d_rho_fx = nullptr;   // rho(k) accumulators (fixed point)
    int* d_kcnt = nullptr;                    // per k tile: chunks done (rho kernel)
    float2* d_kab = nullptr;                  // FP32 force coefficients per k
    double* d_kcoef = nullptr;                // coef_scale / k^2 per k
    bool mh = false;                          // paper's MH sampler (chains in the handle)
    int mh_words = 0;                         // largest 2M+1 (MH tables staged per block)
    uint64_t* d_mh_tq = nullptr;              // MH proposal thresholds, all systems
    double* d_mh_rho = nullptr;               // MH acceptance ratios, all systems
    int4* d_mh_state = nullptr;               // per system: current (m_x, m_y, m_z)
    uint64_t* d_mh_pos = nullptr;             // per system: chain iterations done
    NhState* d_nh = nullptr;                  // per system: Nose-Hoover state
    // neighbour list of the mixed MD step (pairs within r_c + skin)
    bool list = false;                        // the handle keeps a list (skin >= 0)
    bool list_valid = false;                  // sorted arrays still those of the last build
    int list_split = 0, cur_lsplit = -1;      // lanes per particle of the list pass (0 = auto)
    int lsplit = 1, nlblk = 0, max_lblk = 0;
    int list_cap = 0;                         // entries per particle
    Tile* d_lblk = nullptr;
    int* d_nbr = nullptr;                     // [slot * ntot + sorted index]
    int* d_ncnt = nullptr;
    uint4* d_sref = nullptr;
    int* d_iperm = nullptr;
    int* d_list_flag = nullptr;
    unsigned long long* d_list_stats = nullptr;   // builds, largest count
    float4* d_freal = nullptr;                // real-space force of a list step
    // mapped page-locked host words: [0] the step index of a host-buffer
    // call, [1] the device error word read back behind the outputs, [2] the
    // completion word of a zero-copy list step (the step index after it)
    uint64_t* h_pin = nullptr;
    uint64_t* h_pin_dev = nullptr;            // h_pin as the device sees it
    unsigned int* d_done_cnt = nullptr;       // blocks of the closing kernel finished
    cudaEvent_t ev_real = nullptr;            // list step: real-space pass done
    cudaStream_t stream3 = nullptr;           // list step: the rebuild branch
    cudaEvent_t ev_chain = nullptr;           // list step: rebuild branch done
    cudaEvent_t ev_prep = nullptr;            // list step: prep kernel done
    unsigned long long* d_qsum_fx = nullptr;  // sum q per system (fixed point)
    double2* d_blk_e = nullptr;
    double2* d_blk_w = nullptr;               // per real-space block (W_coul, W_lj)
    // observables (allocated on first use): half-space wave vectors per system,
    // their fixed-point structure factors, the real-space virials and the results
    int obs_mmax = -1;
    std::vector<int> obs_off, obs_K;
    int4* d_obs_m = nullptr;
    unsigned long long* d_obs_rho = nullptr;
    double2* d_obs_part = nullptr;            // per-block wave-vector partials
    double* d_obs_w = nullptr;
    double* d_obs_out = nullptr;
    double2* d_blk_q = nullptr;
    uint64_t* d_cur_step = nullptr;
    uint64_t* d_stage_step = nullptr;
    int* d_err = nullptr;
    float4* d_stage_pos = nullptr;
    float4* d_stage_vel = nullptr;
    float4* d_stage_F = nullptr;
    double* d_stage_E = nullptr;
};

namespace {

rbe_status fail(rbe_ctx* h, rbe_status s, const std::string& msg) {
    g_last_error = msg;
    if (h) h->err = msg;
    return s;
}

rbe_status cuda_fail(rbe_ctx* h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, RBE_ERR_CUDA, m);
}

// A host wait ran out (rbe_set_wait_limit): the work stays queued on the stream.
rbe_status timeout_fail(rbe_ctx* h) {
    return fail(h, RBE_ERR_TIMEOUT, "the wait limit passed before the GPU work finished; it is "
                                    "still queued: call rbe_sync before reading or freeing the "
                                    "call's buffers");
}

#define RBE_CUDA(h, call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

// Largest skin that keeps the cell grid (side >= r_c + skin, at least 3 per
// edge) when r_c <= L/3, or the minimum image (r_c + skin <= L/2) in the
// one-cell mode.
double max_skin(const rbe_params& p) {
    return p.box >= 3.0 * p.r_c ? p.box / 3.0 - p.r_c : p.box / 2.0 - p.r_c;
}

// The skin in effect: 0.1 r_c by default, capped as above; 0 for skin < 0.
double skin_of(const rbe_params& p) {
    if (p.skin < 0.0) return 0.0;
    const double s = p.skin > 0.0 ? p.skin : 0.1 * p.r_c;
    return std::max(0.0, std::min(s, max_skin(p)));
}

rbe_status validate_params(const rbe_params& p, std::string& why) {
    if (!(p.box > 0.0) || !std::isfinite(p.box)) { why = "box must be > 0"; return RBE_ERR_ARG; }
    if (!(p.alpha > 0.0) || !std::isfinite(p.alpha)) { why = "alpha must be > 0"; return RBE_ERR_ARG; }
    if (!(p.r_c > 0.0)) { why = "r_c must be > 0"; return RBE_ERR_ARG; }
    if (p.box / p.r_c < 2.0) { why = "r_c must be <= L/2 (minimum image)"; return RBE_ERR_ARG; }
    if (p.P < 1) { why = "P must be >= 1"; return RBE_ERR_ARG; }
    if (p.n_max < 0) { why = "n_max must be >= 0"; return RBE_ERR_ARG; }
    if (p.lj_eps != 0.0) {
        if (!(p.lj_sigma > 0.0) || !(p.lj_rcut > 0.0)) { why = "LJ sigma and cutoff must be > 0"; return RBE_ERR_ARG; }
        if (p.lj_rcut > p.r_c) { why = "lj_rcut must be <= r_c"; return RBE_ERR_ARG; }
    }
    if (!(p.mass > 0.0)) { why = "mass must be > 0"; return RBE_ERR_ARG; }
    if (p.sampler != RBE_SAMPLER_EXACT && p.sampler != RBE_SAMPLER_MH) { why = "sampler must be RBE_SAMPLER_EXACT or RBE_SAMPLER_MH"; return RBE_ERR_ARG; }
    if (p.thermostat != RBE_THERMO_LANGEVIN && p.thermostat != RBE_THERMO_ANDERSEN &&
        p.thermostat != RBE_THERMO_NOSE_HOOVER) { why = "thermostat must be RBE_THERMO_LANGEVIN, RBE_THERMO_ANDERSEN or RBE_THERMO_NOSE_HOOVER"; return RBE_ERR_ARG; }
    if (p.thermostat == RBE_THERMO_NOSE_HOOVER && (!(p.nh_tau > 0.0) || !std::isfinite(p.nh_tau) || !(p.kT > 0.0))) { why = "Nose-Hoover needs nh_tau > 0 and kT > 0"; return RBE_ERR_ARG; }
    if (!(p.andersen_nu >= 0.0) || !(p.andersen_nu * p.dt <= 1.0)) { why = "andersen_nu must satisfy 0 <= nu dt <= 1"; return RBE_ERR_ARG; }
    if (p.gamma < 0.0 || p.kT < 0.0) { why = "gamma and kT must be >= 0"; return RBE_ERR_ARG; }
    if (!std::isfinite(p.skin)) { why = "skin must be finite"; return RBE_ERR_ARG; }
    if (p.skin > 0.0 && p.skin > max_skin(p) * (1.0 + 1e-12)) { why = "skin must be <= L/3 - r_c (L/2 - r_c when r_c > L/3)"; return RBE_ERR_ARG; }
    const int M = axis_M(p.alpha, p.box);
    if (M > 200000) { why = "alpha L^2 too large for the sampling table"; return RBE_ERR_ARG; }
    // (0,0,0) is drawn with probability 1/H^3; keep the 32-attempt loop safe.
    const double H = std::sqrt(p.alpha * p.box * p.box / M_PI);
    if (H * H * H < 2.0) { why = "alpha L^2 too small: k = 0 would dominate the sampler"; return RBE_ERR_ARG; }
    return RBE_OK;
}

void fill_sysdev(const SysHost& s, SysDev& d) {
    const rbe_params& p = s.p;
    const double L = p.box;
    d.L = L;
    d.invL = 1.0 / L;
    d.V = L * L * L;
    d.alpha = p.alpha;
    d.sqrt_alpha = std::sqrt(p.alpha);
    d.r_c = p.r_c;
    d.lB = p.coulomb_prefactor;
    d.S = s.S;
    d.coef_scale = p.coulomb_prefactor * (s.S / (double)p.P) * 4.0 * M_PI / d.V;
    d.self_coef = p.coulomb_prefactor * std::sqrt(p.alpha / M_PI);
    d.bg_coef = p.coulomb_prefactor * M_PI / (d.V * p.alpha);
    d.lj_eps = p.lj_eps;
    d.lj_sigma2 = p.lj_sigma * p.lj_sigma;
    d.lj_rcut2 = p.lj_rcut * p.lj_rcut;
    if (p.lj_eps != 0.0) {
        const double sr6 = std::pow(p.lj_sigma / p.lj_rcut, 6.0);
        d.lj_shift = -4.0 * p.lj_eps * (sr6 * sr6 - sr6);
    } else {
        d.lj_shift = 0.0;
    }
    d.c1 = std::exp(-p.gamma * p.dt / p.mass);
    d.c2 = std::sqrt((1.0 - d.c1 * d.c1) * p.kT / p.mass);
    d.dt = p.dt;
    d.dt_over_m = p.dt / p.mass;
    const double scale = 4294967296.0 / L;
    d.fx_hi = (float)scale;
    d.fx_lo = (float)(scale - (double)d.fx_hi);
    d.Lf = (float)L;
    d.L_over_2_32 = (float)(L / 4294967296.0);
    d.seed = p.seed;
    d.stream = p.stream;
    d.n = s.n;
    d.P = p.P;
    d.M = s.M;
    d.ncd = s.ncd;
    d.off_p = s.off_p;
    d.off_c = s.off_c;
    d.off_k = s.off_k;
    d.off_t = s.off_t;
    d.off_part = 0;
    d.nchunk = 0;
    d.off_b = 0;
    d.nb = 0;
    d.off_rb = 0;
    d.nrb = 0;
    d.off_sg = 0;
    d.nsg = 0;
    d.off_lb = 0;
    d.nlb = 0;
    // rho(k) accumulators: |rho| <= sum |q| <= 4 n is assumed; the largest
    // power of two (at most 2^52) that keeps 4 n * scale below 2^62.
    int e = 52;
    const double bound = 4.0 * std::max(1, s.n);
    while (e > 20 && bound * std::ldexp(1.0, e) >= std::ldexp(1.0, 62)) --e;
    d.rho_scale = std::ldexp(1.0, e);
    d.rho_inv_scale = std::ldexp(1.0, -e);
    d.f_rc2 = (float)(d.r_c * d.r_c);
    d.f_lj_rc2 = (float)d.lj_rcut2;
    d.f_alpha = (float)d.alpha;
    d.f_sqrt_alpha = (float)d.sqrt_alpha;
    d.f_two_sa_spi = (float)(2.0 * d.sqrt_alpha / std::sqrt(M_PI));
    d.f_lB = (float)d.lB;
    d.f_lj_sigma2 = (float)d.lj_sigma2;
    d.f_lj_eps = (float)d.lj_eps;
    d.f_lj_shift = (float)d.lj_shift;
    d.f_c1 = (float)d.c1;
    d.f_c2 = (float)d.c2;
    d.f_dt = (float)d.dt;
    d.f_dt_over_m = (float)d.dt_over_m;
    d.f_invL = (float)d.invL;
    d.thermostat = p.thermostat;
    {
        double thr = std::floor(p.andersen_nu * p.dt * 4294967296.0);
        d.andersen_thr = (uint64_t)std::min(thr, 4294967296.0);
    }
    d.vsd = std::sqrt(p.kT / p.mass);
    d.f_vsd = (float)d.vsd;
    d.f_inv_Lu = (float)(4294967296.0 / L);
    d.nh_rate = p.thermostat == RBE_THERMO_NOSE_HOOVER
                    ? p.dt / (3.0 * std::max(1, s.n) * p.nh_tau * p.nh_tau) : 0.0;
    d.nh_k2scale = p.kT > 0.0 ? p.mass / p.kT * 4294967296.0 : 0.0;
    d.f_list_cut2 = (float)((p.r_c + s.skin) * (p.r_c + s.skin) * (1.0 + 1e-5));
    d.f_half_skin2 = (float)(0.25 * s.skin * s.skin * (1.0 - 1e-5));
    d.corner_q = (uint32_t)(4294967296ull / (unsigned long long)std::max(1, s.ncd));
    d.corner_r = (uint32_t)(4294967296ull - (unsigned long long)d.corner_q * std::max(1, s.ncd));
}

// Smallest system (particles over all replicas) that fuses the structure
// factors with the standing-list pass when no autotune has chosen: one launch
// of both kinds of block gains once each kind alone fills the GPU (2^20: 0.58
// against 0.62 ms per step; 2^18: 0.176 against 0.172 ms).
constexpr long long kFuseMinN = 1LL << 19;

bool fusion_on(const rbe_ctx* h) {
    if (h->fusion_mode >= 0) return h->fusion_mode == 1;
    if (h->fuse_tuned >= 0) return h->fuse_tuned == 1;
    const long long ntot = h->batch ? h->ntot : std::max(h->cur_n, 0);
    return ntot >= kFuseMinN;
}

int auto_chunk(const rbe_ctx* h, long long ntot) {
    const int ltiles = (h->pmax + kRhoKT - 1) / kRhoKT;
    const long long target_blocks = 152LL * 12;
    long long chunks = std::max(1LL, target_blocks / std::max(1, ltiles));
    long long c = (ntot + chunks - 1) / chunks;
    int p = pow2_ceil(std::max(1LL, c));
    return std::min(4096, std::max(32, p));
}

int auto_split(long long ntot) {
    const long long target_threads = 152LL * 8 * kBlockP;
    int s = 1;
    while (s < 8 && ntot * s < target_threads) s <<= 1;
    return s;
}

// Threads per particle of the mixed real-space pass (each takes 9/R of the 9
// neighbour rows): 9 while that still leaves few threads per SM, else 3.
int auto_real_split(long long ntot) {
    return ntot * 9 <= 152LL * 4096 ? 9 : 3;
}

// Threads per particle of the neighbour-list pass: enough for about 1024
// threads per SM.
int auto_list_split(long long ntot) {
    int r = 1;
    while (r < 8 && ntot * r < 152LL * 1024) r <<= 1;
    return r;
}

// Threads per particle of the FP64 real-space pass: the largest power of two
// not above the mixed path's.
int real_split64(int r) { return r >= 8 ? 8 : (r >= 2 ? 2 : 1); }

// Cells along x per real-space block: enough blocks to fill the GPU, and a
// staged neighbourhood (9 rows of seg + 2 cells) of about 2500 records.
int auto_real_seg(long long ntot, long long ncell, int ncd) {
    const double occ = ncell > 0 ? (double)ntot / (double)ncell : 1.0;
    int seg = (int)std::floor(2500.0 / (9.0 * std::max(occ, 0.5)) - 2.0);
    const long long min_blocks = 152LL * 4;
    seg = std::min(seg, (int)std::max(1LL, ncell / min_blocks));
    return std::max(1, std::min(seg, ncd));
}

// (Re)build the work tables for the current particle counts and tuning.
rbe_status prepare(rbe_ctx* h, int n) {
    if (!h->batch) h->sys[0].n = n;
    const long long ntot = h->batch ? h->ntot : n;
    const int chunk = h->rho_chunk > 0 ? h->rho_chunk : auto_chunk(h, ntot);
    const int split = h->force_split > 0 ? h->force_split : auto_split(ntot);
    const int rsplit = h->real_split > 0 ? h->real_split : auto_real_split(ntot);
    const int lsplit = h->list_split > 0 ? h->list_split : auto_list_split(ntot);
    int ncd_max = 3;
    for (auto& sh : h->sys) ncd_max = std::max(ncd_max, sh.ncd);
    const int rseg = h->real_seg > 0 ? std::min(h->real_seg, ncd_max)
                                     : auto_real_seg(ntot, h->ncell, ncd_max);
    if (h->cur_n == n && h->cur_chunk == chunk && h->cur_split == split &&
        h->cur_rsplit == rsplit && h->cur_seg == rseg && h->cur_lsplit == lsplit)
        return RBE_OK;
    h->list_valid = false;                 // the sorted arrays are rebuilt from scratch
    std::vector<Tile> segs;
    int seg_max = 1;
    double stage_need = 0.0;
    std::vector<Tile> pblk, fblk, rblk, chunks, lblk;
    const int ltile = kBlockP / lsplit;
    const int ftile = kBlockP / split;
    const int rtile = kBlockP / real_split64(rsplit);
    int off_part = 0;
    for (int s = 0; s < h->nsys; ++s) {
        SysHost& sh = h->sys[s];
        SysDev& d = h->sysdev[s];
        fill_sysdev(sh, d);
        d.off_b = (int)pblk.size();
        int nb = 0;
        for (int f = 0; f < sh.n || (f == 0 && nb == 0); f += kBlockP) {
            pblk.push_back(Tile{s, sh.off_p + f, std::min(kBlockP, sh.n - f), 0});
            ++nb;
            if (sh.n == 0) break;
        }
        d.nb = nb;
        for (int f = 0; f < sh.n || f == 0; f += ftile) {
            fblk.push_back(Tile{s, sh.off_p + f, std::max(0, std::min(ftile, sh.n - f)), 0});
            if (sh.n == 0) break;
        }
        d.off_rb = (int)rblk.size();
        int nrb = 0;
        for (int f = 0; f < sh.n || f == 0; f += rtile) {
            rblk.push_back(Tile{s, sh.off_p + f, std::max(0, std::min(rtile, sh.n - f)), 0});
            ++nrb;
            if (sh.n == 0) break;
        }
        d.nrb = nrb;
        d.off_lb = (int)lblk.size();
        if (h->list)
            for (int f = 0; f < sh.n || f == 0; f += ltile) {
                lblk.push_back(Tile{s, sh.off_p + f, std::max(0, std::min(ltile, sh.n - f)), 0});
                if (sh.n == 0) break;
            }
        d.nlb = (int)lblk.size() - d.off_lb;
        d.off_sg = (int)segs.size();
        {
            const int ncd = sh.ncd, seg = std::min(rseg, ncd);
            for (int z = 0; z < ncd; ++z)
                for (int y = 0; y < ncd; ++y)
                    for (int x0 = 0; x0 < ncd; x0 += seg) {
                        const int cnt = std::min(seg, ncd - x0);
                        segs.push_back(Tile{s, sh.off_c + (z * ncd + y) * ncd + x0, cnt,
                                            x0 | (y << 10) | (z << 20)});
                        seg_max = std::max(seg_max, cnt);
                    }
            const double occ = (double)sh.n / ((double)ncd * ncd * ncd);
            const double mean = 9.0 * (seg + 2) * occ;
            stage_need = std::max(stage_need, mean + 6.0 * std::sqrt(mean) + 64.0);
        }
        d.nsg = (int)segs.size() - d.off_sg;
        d.off_part = off_part;
        int nc = 0;
        for (int f = 0; f < sh.n || f == 0; f += chunk) {
            chunks.push_back(Tile{s, sh.off_p + f, std::max(0, std::min(chunk, sh.n - f)), nc});
            ++nc;
            if (sh.n == 0) break;
        }
        d.nchunk = nc;
        off_part += nc * sh.p.P;
    }
    if ((int)pblk.size() > h->max_pblk || (int)fblk.size() > h->max_fblk ||
        (int)rblk.size() > h->max_rblk || (int)chunks.size() > h->max_chunks ||
        (int)segs.size() > h->max_seg || (int)lblk.size() > h->max_lblk ||
        (size_t)off_part > h->max_part)
        return fail(h, RBE_ERR_ARG, "work tables exceed the workspace (n > capacity?)");
    RBE_CUDA(h, cudaMemcpyAsync(h->d_sys, h->sysdev.data(), sizeof(SysDev) * h->nsys,
                                cudaMemcpyHostToDevice, h->stream));
    RBE_CUDA(h, cudaMemcpyAsync(h->d_pblk, pblk.data(), sizeof(Tile) * pblk.size(),
                                cudaMemcpyHostToDevice, h->stream));
    RBE_CUDA(h, cudaMemcpyAsync(h->d_fblk, fblk.data(), sizeof(Tile) * fblk.size(),
                                cudaMemcpyHostToDevice, h->stream));
    RBE_CUDA(h, cudaMemcpyAsync(h->d_rblk, rblk.data(), sizeof(Tile) * rblk.size(),
                                cudaMemcpyHostToDevice, h->stream));
    RBE_CUDA(h, cudaMemcpyAsync(h->d_segs, segs.data(), sizeof(Tile) * segs.size(),
                                cudaMemcpyHostToDevice, h->stream));
    RBE_CUDA(h, cudaMemcpyAsync(h->d_chunks, chunks.data(), sizeof(Tile) * chunks.size(),
                                cudaMemcpyHostToDevice, h->stream));
    if (!lblk.empty())
        RBE_CUDA(h, cudaMemcpyAsync(h->d_lblk, lblk.data(), sizeof(Tile) * lblk.size(),
                                    cudaMemcpyHostToDevice, h->stream));
    h->nlblk = (int)lblk.size();
    h->lsplit = lsplit;
    RBE_CUDA(h, cudaStreamSynchronize(h->stream));
    h->npblk = (int)pblk.size();
    h->nfblk = (int)fblk.size();
    h->nrblk = (int)rblk.size();
    h->nchunks = (int)chunks.size();
    h->split = split;
    h->rsplit = rsplit;
    h->nseg = (int)segs.size();
    h->seg_max = seg_max;
    // staged records per segment block: the expected neighbourhood plus six
    // standard deviations, within a 96 KB budget (larger ones read global memory)
    h->stage_cap = (int)std::min(6144.0, std::ceil(stage_need));
    {
        // warps of 32 / rsplit particles, enough for a segment two standard
        // deviations above the mean in one pass (a fuller segment makes a
        // second pass and stretches the kernel's tail)
        const double per_seg = (double)std::max<long long>(ntot, 1) * seg_max /
                               std::max(1, h->ncell);
        const double want = 32.0 * std::ceil((per_seg + 2.0 * std::sqrt(per_seg)) /
                                             (32 / rsplit));
        h->seg_threads = want > 192 ? 256 : (want > 128 ? 192 : (want > 64 ? 128 : 64));
    }
    h->cur_seg = rseg;
    h->cur_n = n;
    h->cur_chunk = chunk;
    h->cur_split = split;
    h->cur_rsplit = rsplit;
    h->cur_lsplit = lsplit;
    return RBE_OK;
}

rbe_status allocate(rbe_ctx* h) {
    // capacities (chunks as small as 32 particles, force tiles as small as 16)
    long long pb = 0, fb = 0, rb = 0, ch = 0, part = 0;
    for (auto& s : h->sys) {
        const long long n = h->batch ? s.n : s.p.n_max;
        pb += (n + kBlockP - 1) / kBlockP + 1;
        fb += (n + 15) / 16 + 1;
        rb += (n + 3) / 4 + 1;
        const long long c = (n + 31) / 32 + 1;
        ch += c;
        part += c * s.p.P;
    }
    h->max_pblk = (int)pb;
    h->max_lblk = (int)(pb * 8);             // list tiles as small as kBlockP / 8
    h->max_fblk = (int)fb;
    h->max_rblk = (int)rb;
    h->max_seg = std::max(1, h->ncell);
    h->max_chunks = (int)ch;
    h->max_part = (size_t)part;
    const size_t N = (size_t)std::max(h->ntot, 1);
    rbe_status st = RBE_OK;
#define RBE_ALLOC(ptr, cnt) \
    if ((st = dalloc(&(ptr), (size_t)(cnt))) != RBE_OK) return fail(h, st, "cudaMalloc failed: " #ptr)
    RBE_ALLOC(h->d_sys, h->nsys);
    RBE_ALLOC(h->d_pblk, pb);
    RBE_ALLOC(h->d_fblk, fb);
    RBE_ALLOC(h->d_rblk, rb);
    RBE_ALLOC(h->d_segs, std::max(1, h->ncell));
    RBE_ALLOC(h->d_chunks, ch);
    RBE_ALLOC(h->d_kstart, h->nsys + 1);
    RBE_ALLOC(h->d_cstart, h->nsys + 1);
    RBE_ALLOC(h->d_table, h->ttot);
    RBE_ALLOC(h->d_fx, N);
    RBE_ALLOC(h->d_spos, N);
    RBE_ALLOC(h->d_fx64, N);
    RBE_ALLOC(h->d_spos64, N);
    RBE_ALLOC(h->d_cid, N);
    RBE_ALLOC(h->d_rank, N);
    RBE_ALLOC(h->d_perm, N);
    RBE_ALLOC(h->d_perm_tmp, N);
    RBE_ALLOC(h->d_fs, N);
    RBE_ALLOC(h->d_fs64, N);
    RBE_ALLOC(h->d_cell_cnt, h->ncell + 1);
    RBE_ALLOC(h->d_cell_start, h->ncell + 1);
    RBE_ALLOC(h->d_ksamp, h->ktot);
    RBE_ALLOC(h->d_rho_fx, 2 * (size_t)h->ktot);
    RBE_ALLOC(h->d_kcnt, h->ktot);
    RBE_ALLOC(h->d_kcoef, h->ktot);
    RBE_ALLOC(h->d_mh_tq, h->ttot);
    RBE_ALLOC(h->d_mh_rho, h->ttot);
    RBE_ALLOC(h->d_mh_state, h->nsys);
    RBE_ALLOC(h->d_mh_pos, h->nsys);
    RBE_ALLOC(h->d_nh, h->nsys);
    if (h->list) {
        RBE_ALLOC(h->d_lblk, h->max_lblk);
        RBE_ALLOC(h->d_nbr, (size_t)h->list_cap * N);
        RBE_ALLOC(h->d_ncnt, N);
        RBE_ALLOC(h->d_sref, N);
        RBE_ALLOC(h->d_iperm, N);
        RBE_ALLOC(h->d_list_flag, 1);
        RBE_ALLOC(h->d_list_stats, 2);
        RBE_ALLOC(h->d_freal, N);
    }
    RBE_ALLOC(h->d_kab, h->ktot);
    RBE_ALLOC(h->d_qsum_fx, h->nsys);
    // per-block energy / virial partials: FP64 blocks, segment blocks or list blocks
    const long long nblk_e = std::max<long long>(std::max<long long>(rb, (long long)kSegChunks *
                                                 (h->ncell + 1)), (long long)h->max_lblk);
    RBE_ALLOC(h->d_blk_e, nblk_e);
    RBE_ALLOC(h->d_blk_w, nblk_e);
    RBE_ALLOC(h->d_blk_q, pb);
    RBE_ALLOC(h->d_cur_step, 1);
    RBE_ALLOC(h->d_stage_step, 1);
    RBE_ALLOC(h->d_err, 1);
    RBE_ALLOC(h->d_stage_pos, N);
    RBE_ALLOC(h->d_stage_vel, N);
    RBE_ALLOC(h->d_stage_F, N);
    RBE_ALLOC(h->d_stage_E, 4 * h->nsys);
#undef RBE_ALLOC
    RBE_CUDA(h, cudaMemset(h->d_cell_cnt, 0, sizeof(int) * (h->ncell + 1)));
    RBE_CUDA(h, cudaMemset(h->d_err, 0, sizeof(int)));
    if (h->list) {
        // sorted slots 0 until the first build (which the set flag forces); list
        // slots always hold valid indices (the list pass loads ahead of counts)
        RBE_CUDA(h, cudaMemset(h->d_iperm, 0, sizeof(int) * N));
        RBE_CUDA(h, cudaMemset(h->d_nbr, 0, sizeof(int) * (size_t)h->list_cap * N));
        RBE_CUDA(h, cudaMemset(h->d_ncnt, 0, sizeof(int) * N));
        RBE_CUDA(h, cudaMemset(h->d_sref, 0, sizeof(uint4) * N));
        RBE_CUDA(h, cudaMemset(h->d_list_stats, 0, sizeof(unsigned long long) * 2));
        const int one = 1;
        RBE_CUDA(h, cudaMemcpy(h->d_list_flag, &one, sizeof(int), cudaMemcpyHostToDevice));
    }
    RBE_CUDA(h, cudaMemset(h->d_qsum_fx, 0, sizeof(unsigned long long) * h->nsys));
    RBE_CUDA(h, cudaMemset(h->d_rho_fx, 0, sizeof(unsigned long long) * 2 * h->ktot));
    RBE_CUDA(h, cudaMemset(h->d_kcnt, 0, sizeof(int) * h->ktot));
    std::vector<uint64_t> tab, mtq;
    std::vector<double> mrho;
    std::vector<int> kstart, cstart;
    for (auto& s : h->sys) {
        tab.insert(tab.end(), s.table.begin(), s.table.end());
        mtq.insert(mtq.end(), s.mh_tq.begin(), s.mh_tq.end());
        mrho.insert(mrho.end(), s.mh_rho.begin(), s.mh_rho.end());
        kstart.push_back(s.off_k);
        cstart.push_back(s.off_c);
    }
    kstart.push_back(h->ktot);
    cstart.push_back(h->ncell);
    RBE_CUDA(h, cudaMemcpy(h->d_cstart, cstart.data(), sizeof(int) * cstart.size(),
                           cudaMemcpyHostToDevice));
    RBE_CUDA(h, cudaMemcpy(h->d_table, tab.data(), sizeof(uint64_t) * tab.size(),
                           cudaMemcpyHostToDevice));
    RBE_CUDA(h, cudaMemcpy(h->d_kstart, kstart.data(), sizeof(int) * kstart.size(),
                           cudaMemcpyHostToDevice));
    RBE_CUDA(h, cudaMemcpy(h->d_mh_tq, mtq.data(), sizeof(uint64_t) * mtq.size(),
                           cudaMemcpyHostToDevice));
    RBE_CUDA(h, cudaMemcpy(h->d_mh_rho, mrho.data(), sizeof(double) * mrho.size(),
                           cudaMemcpyHostToDevice));
    RBE_CUDA(h, cudaMemset(h->d_mh_state, 0, sizeof(int4) * h->nsys));   // chains start at m = 0
    RBE_CUDA(h, cudaMemset(h->d_mh_pos, 0, sizeof(uint64_t) * h->nsys));
    {
        std::vector<NhState> nh(h->nsys);             // xi = 0, kept on the first step
        for (auto& v : nh) {
            v = NhState{};
            v.first = 1;
        }
        RBE_CUDA(h, cudaMemcpy(h->d_nh, nh.data(), sizeof(NhState) * h->nsys,
                               cudaMemcpyHostToDevice));
    }
    RBE_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    RBE_CUDA(h, cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking));
    RBE_CUDA(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    RBE_CUDA(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    RBE_CUDA(h, cudaEventCreateWithFlags(&h->ev_real, cudaEventDisableTiming));
    RBE_CUDA(h, cudaEventCreateWithFlags(&h->ev_chain, cudaEventDisableTiming));
    RBE_CUDA(h, cudaEventCreateWithFlags(&h->ev_prep, cudaEventDisableTiming));
    RBE_CUDA(h, cudaStreamCreateWithFlags(&h->stream3, cudaStreamNonBlocking));
    RBE_CUDA(h, cudaHostAlloc((void**)&h->h_pin, 4 * sizeof(uint64_t), cudaHostAllocMapped));
    h->h_pin[0] = h->h_pin[1] = h->h_pin[2] = h->h_pin[3] = 0;
    RBE_CUDA(h, cudaHostGetDevicePointer((void**)&h->h_pin_dev, h->h_pin, 0));
    RBE_CUDA(h, cudaMalloc(&h->d_done_cnt, sizeof(unsigned int)));
    RBE_CUDA(h, cudaMemset(h->d_done_cnt, 0, sizeof(unsigned int)));
    return RBE_OK;
}

void release(rbe_ctx* h) {
    if (!h) return;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    void* ptrs[] = {h->d_sys, h->d_pblk, h->d_fblk, h->d_rblk, h->d_segs, h->d_chunks,
                    h->d_kstart,
                    h->d_cstart,
                    h->d_table, h->d_fx, h->d_spos, h->d_fx64, h->d_spos64, h->d_cid, h->d_rank,
                    h->d_perm, h->d_perm_tmp, h->d_fs, h->d_fs64, h->d_cell_cnt,
                    h->d_cell_start, h->d_ksamp, h->d_rho_fx, h->d_kcnt, h->d_kab,
                    h->d_kcoef, h->d_mh_tq, h->d_mh_rho, h->d_mh_state, h->d_mh_pos, h->d_nh,
                    h->d_lblk, h->d_nbr, h->d_ncnt, h->d_sref, h->d_iperm, h->d_list_flag,
                    h->d_list_stats, h->d_freal,
                    h->d_qsum_fx, h->d_blk_e, h->d_blk_w, h->d_obs_m, h->d_obs_rho, h->d_obs_w,
                    h->d_obs_out, h->d_obs_part, h->d_blk_q, h->d_cur_step, h->d_stage_step,
                    h->d_err, h->d_stage_pos, h->d_stage_vel, h->d_stage_F, h->d_stage_E,
                    h->d_done_cnt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_real) cudaEventDestroy(h->ev_real);
    if (h->ev_chain) cudaEventDestroy(h->ev_chain);
    if (h->ev_prep) cudaEventDestroy(h->ev_prep);
    if (h->stream3) cudaStreamDestroy(h->stream3);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    for (int k = 0; k < RBE_K_COUNT; ++k) {
        if (h->ev_beg[k]) cudaEventDestroy(h->ev_beg[k]);
        if (h->ev_end[k]) cudaEventDestroy(h->ev_end[k]);
    }
}

rbe_status create_common(const rbe_params* ps, const int32_t* ns, int nsys, bool batch,
                         rbe_handle* out) {
    if (!out) return fail(nullptr, RBE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ps || nsys < 1) return fail(nullptr, RBE_ERR_ARG, "no systems");
    rbe_ctx* h = new rbe_ctx();
    h->batch = batch;
    h->nsys = nsys;
    h->sys.resize(nsys);
    h->sysdev.resize(nsys);
    int off_p = 0, off_c = 0, off_k = 0, off_t = 0;
    for (int s = 0; s < nsys; ++s) {
        SysHost& sh = h->sys[s];
        sh.p = ps[s];
        std::string why;
        if (validate_params(sh.p, why) != RBE_OK) {
            rbe_status st = fail(nullptr, RBE_ERR_ARG, "system " + std::to_string(s) + ": " + why);
            delete h;
            return st;
        }
        sh.n = batch ? ns[s] : sh.p.n_max;
        if (batch && ns[s] < 0) {
            delete h;
            return fail(nullptr, RBE_ERR_ARG, "negative particle count");
        }
        sh.M = axis_M(sh.p.alpha, sh.p.box);
        sh.H = build_table(sh.p.alpha, sh.p.box, sh.M, sh.table);
        build_mh_tables(sh.p.alpha, sh.p.box, sh.M, sh.mh_tq, sh.mh_rho);
        if (sh.p.sampler != ps[0].sampler) {
            delete h;
            return fail(nullptr, RBE_ERR_ARG, "all systems of a handle must use the same sampler");
        }
        sh.S = sh.H * sh.H * sh.H - 1.0;
        // cells of side >= r_c + skin, at least 3 per edge; else one cell (all pairs)
        sh.skin = skin_of(sh.p);
        const double side = sh.p.r_c + sh.skin;
        sh.ncd = sh.p.box / side >= 3.0 ? std::min(256, (int)std::floor(sh.p.box / side)) : 1;
        if ((sh.p.skin < 0.0) != (ps[0].skin < 0.0)) {
            delete h;
            return fail(nullptr, RBE_ERR_ARG, "all systems of a handle must agree on skin < 0");
        }
        sh.off_p = off_p;
        sh.off_c = off_c;
        sh.off_k = off_k;
        sh.off_t = off_t;
        off_p += sh.n;
        off_c += sh.ncd * sh.ncd * sh.ncd;
        off_k += sh.p.P;
        off_t += 2 * sh.M + 1;
        h->pmax = std::max(h->pmax, sh.p.P);
    }
    h->ntot = off_p;
    h->ncell = off_c;
    h->ktot = off_k;
    h->ttot = off_t;
    h->mh = ps[0].sampler == RBE_SAMPLER_MH;
    h->list = ps[0].skin >= 0.0;
    if (h->list) {
        // entries per particle: the mean count within r_c + skin at the
        // system's density, plus 50 % and eight standard deviations
        double most = 0.0;
        for (auto& sh : h->sys) {
            const double rr = sh.p.r_c + sh.skin;
            const double nn = batch ? sh.n : sh.p.n_max;
            most = std::max(most, 4.0 / 3.0 * M_PI * rr * rr * rr * nn /
                                      (sh.p.box * sh.p.box * sh.p.box));
        }
        h->list_cap = (int)std::min(4096.0, 8.0 * std::ceil((1.5 * most + 8.0 * std::sqrt(most) + 16.0) / 8.0));
    }
    for (auto& sh : h->sys) h->mh_words = std::max(h->mh_words, 2 * sh.M + 1);
    rbe_status st = allocate(h);
    if (st != RBE_OK) {
        std::string m = h->err;
        release(h);
        delete h;
        return fail(nullptr, st, m);
    }
    *out = h;
    return RBE_OK;
}

// Enqueue one evaluation (and optionally one Langevin step) on stream st.
struct EvalArgs {
    int prec;                 // RBE_MIXED or RBE_FP64
    int parts;
    const float4* pos;        // mixed input
    const double4* pos64;     // fp64 input
    uint64_t step;
    uint64_t* step_dev;       // nullable: device step counter (incremented)
    float4* F;
    double4* F64;
    double* E;
    double* W;                // nullable: real-space Coulomb and LJ virials (2 per system)
    float* phi;
    double* phi64;
    float4* md_pos;
    float4* md_vel;
    double4* md_pos64;
    double4* md_vel64;
    bool list;                // mixed MD step over the neighbour list
    bool list_forces;         // mixed forces call over the neighbour list
    unsigned long long* done; // list step, nullable: completion word (mapped host memory)
};

// Kernel work descriptor: tables for a batch, by-value constants and a tile
// size for a single system.
Work make_work(const rbe_ctx* h, const Tile* tiles, int tile, int aux_stride) {
    Work w{};
    if (h->batch) {
        w.sysv = h->d_sys;
        w.tiles = tiles;
    } else {
        w.tile = tile;
        w.aux_stride = aux_stride;
        w.one = h->sysdev[0];
    }
    return w;
}

RealArgs make_real_args(const rbe_ctx* h, int parts) {
    RealArgs r{};
    r.w = make_work(h, h->d_rblk, kBlockP / real_split64(h->rsplit), 0);
    r.nrblk = h->nrblk;
    r.split = h->rsplit;
    r.split64 = real_split64(h->rsplit);
    r.ncell = h->ncell;
    r.nsys = h->nsys;
    r.cstart = h->d_cstart;
    r.segs = h->d_segs;
    r.nseg = h->nseg;
    r.seg_max = h->seg_max;
    r.stage_cap = h->stage_cap;
    r.seg_threads = h->seg_threads;
    r.parts = parts;
    r.cell_start = h->d_cell_start;
    r.perm = h->d_perm;
    r.cur_step = h->d_cur_step;
    r.qsum_fx = h->d_qsum_fx;
    r.spos = h->d_spos;
    r.fs = h->d_fs;
    r.spos64 = h->d_spos64;
    r.fs64 = h->d_fs64;
    r.err = h->d_err;
    return r;
}

// Structure factors: per-chunk partials added to the fixed-point rho(k).
void launch_rho(const rbe_ctx* h, cudaStream_t st, bool mixed, bool pdl = false) {
    const bool one = !h->batch;
    const int kt = mixed ? kRhoKT : kLTile;           // wave vectors per tile
    const int ltiles = (h->pmax + kt - 1) / kt;
    const Work w = make_work(h, h->d_chunks, h->cur_chunk, 1);
    if (mixed)
        launch_rho_mixed(st, one, w, h->nchunks, ltiles, h->d_ksamp, h->d_kcoef, h->d_fx,
                         h->d_rho_fx, h->d_kcnt, h->d_kab, pdl);
    else
        launch_rho_f64(st, one, w, h->nchunks, ltiles, h->d_ksamp, h->d_fx64, h->d_rho_fx);
}

void launch_force(const rbe_ctx* h, cudaStream_t st, bool mixed, const MdOut& md = MdOut{},
                  bool pdl = false) {
    const bool one = !h->batch;
    if (mixed) {
        const Work w = make_work(h, h->split == 1 ? h->d_pblk : h->d_fblk, kBlockP / h->split, 0);
        launch_fourier_force_mixed(st, one, w, h->split == 1 ? h->npblk : h->nfblk, h->split,
                                   h->d_fx, h->d_ksamp, h->d_kab, h->d_fs, md, pdl);
    } else {
        const Work w = make_work(h, h->d_pblk, kBlockP, 0);
        launch_fourier_force_f64(st, one, w, h->npblk, h->d_fx64, h->d_ksamp, h->d_rho_fx,
                                 h->d_fs64);
    }
}

// Returns the number of kernels enqueued.  The Fourier branch (structure
// factors -> finalize -> Fourier force, on the unsorted records) runs on a
// second stream concurrently with the cell-list branch (scan -> scatter ->
// order); both join before the real-space kernel.  With profiling on (and st
// the handle's own stream, i.e. not capturing) every kernel is bracketed by
// events and the per-kernel device times are accumulated after the last one.
int enqueue_eval(rbe_ctx* h, cudaStream_t st, const EvalArgs& a) {
    const bool mixed = a.prec == RBE_MIXED;
    const bool one = !h->batch;
    const bool fourier = (a.parts & RBE_PART_FOURIER) != 0;
    const int want_q = (fourier && (a.E || a.phi || a.phi64)) ? 1 : 0;
    const int n = h->batch ? h->ntot : h->cur_n;
    const bool prof = h->prof_on && st == h->stream;
    // profiling runs the branches one after another on st, so that each
    // kernel's event pair brackets that kernel alone
    cudaStream_t st2 = prof ? st : h->stream2;
    // a list step's structure factors and standing-list pass share one launch
    // (timed as RBE_K_RHO_LIST when profiling)
    const bool fused = a.list && mixed && (a.parts & RBE_PART_FOURIER) && fusion_on(h);
    bool used[RBE_K_COUNT] = {};
    int count = 0;
    auto run = [&](int kid, cudaStream_t s, auto&& launch) {
        if (prof) cudaEventRecord(h->ev_beg[kid], s);
        launch();
        if (prof) {
            cudaEventRecord(h->ev_end[kid], s);
            used[kid] = true;
        }
        ++count;
    };
    const Work wp = make_work(h, h->d_pblk, kBlockP, 0);
    PrepArgs pa{};
    pa.blk_q = h->d_blk_q;
    pa.want_q = want_q;
    pa.qsum_fx = h->d_qsum_fx;
    pa.rho_fx = h->d_rho_fx;
    pa.nrho = h->ktot;
    pa.step_dev = a.step_dev;
    pa.step_arg = a.step;
    pa.cur_step = h->d_cur_step;
    pa.npblk = h->npblk;
    pa.ktot = fourier ? h->ktot : 0;
    pa.nsys = h->nsys;
    pa.kstart = h->d_kstart;
    pa.table = h->d_table;
    pa.tab_words = h->ttot <= 8192 ? h->ttot : 0;    // 32 KB of shared memory at most
    pa.mh = h->mh ? 1 : 0;
    pa.mh_words = h->mh_words;
    pa.mh_tq = h->d_mh_tq;
    pa.mh_rho = h->d_mh_rho;
    pa.mh_state = h->d_mh_state;
    pa.mh_pos = h->d_mh_pos;
    pa.ksamp = h->d_ksamp;
    pa.kcoef = h->d_kcoef;
    pa.err = h->d_err;
    pa.ncell = h->ncell;
    pa.ntot = n;
    pa.nh = (a.md_pos || a.md_pos64) ? h->d_nh : nullptr;
    const bool lst = a.list || a.list_forces;     // the evaluation keeps the list
    if (lst) {
        pa.sref = h->d_sref;
        pa.iperm = h->d_iperm;
        pa.spos = h->d_spos;
        pa.list_flag = h->d_list_flag;
    } else {
        h->list_valid = false;              // the sorted arrays are about to change
    }
    const int* lflag = lst ? h->d_list_flag : nullptr;
    if (want_q)
        cudaMemsetAsync(h->d_qsum_fx, 0, sizeof(unsigned long long) * h->nsys, st);
    run(RBE_K_PREP, st, [&] {
        if (mixed)
            launch_prep_mixed(st, one, wp, h->npblk, a.pos, h->d_fx, h->d_cid, h->d_rank,
                              h->d_cell_cnt, pa);
        else
            launch_prep_f64(st, one, wp, h->npblk, a.pos64, h->d_fx64, h->d_cid, h->d_rank,
                            h->d_cell_cnt, pa);
    });
    if (a.list) {
        // list step: prep -> structure factors -> Fourier force on st with
        // programmatic dependent launches (each kernel's blocks are scheduled
        // while the previous one drains); the list pass and the rebuild fork
        // off after prep
        cudaEventRecord(h->ev_prep, st);
        if (fused) {
            // the structure factors and the pass over a standing list in one
            // launch whose blocks take either kind of work
            RealArgs rl = make_real_args(h, a.parts);
            rl.lw = make_work(h, h->d_lblk, kBlockP / h->lsplit, 0);
            rl.nlblk = h->nlblk;
            rl.lsplit = h->lsplit;
            rl.nbr = h->d_nbr;
            rl.ncnt = h->d_ncnt;
            rl.nbr_stride = std::max(h->ntot, 1);
            rl.nbr_cap = h->list_cap;
            rl.list_flag = h->d_list_flag;
            rl.freal = h->d_freal;
            rl.list_when = 0;
            const int ltiles = (h->pmax + kRhoKT - 1) / kRhoKT;
            run(RBE_K_RHO_LIST, st, [&] {
                launch_rho_list(st, one, make_work(h, h->d_chunks, h->cur_chunk, 1), h->nchunks,
                                ltiles, h->d_ksamp, h->d_kcoef, h->d_fx, h->d_rho_fx, h->d_kcnt,
                                h->d_kab, rl, !prof);
            });
        } else if (fourier) {
            run(RBE_K_RHO, st, [&] { launch_rho(h, st, mixed, !prof); });
        }
    } else if (fourier) {
        cudaEventRecord(h->ev_fork, st);
        cudaStreamWaitEvent(st2, h->ev_fork, 0);
        run(RBE_K_RHO, st2, [&] { launch_rho(h, st2, mixed); });
        run(RBE_K_FOURIER_FORCE, st2, [&] { launch_force(h, st2, mixed); });
        cudaEventRecord(h->ev_join, st2);
    }
    // the cell list; on a list step the (usually no-op) rebuild runs on a
    // third stream, so that the list pass need not wait for it
    cudaStream_t sc = st;
    if (a.list) {
        sc = prof ? st : h->stream3;
        cudaStreamWaitEvent(sc, h->ev_prep, 0);
    }
    run(RBE_K_SCAN, sc, [&] {
        // on a list evaluation the cells are assigned here, only for a rebuild
        // (the prep kernel skips them): counted with the scan in the profile
        if (lst && mixed) {
            launch_cell_assign(sc, one, wp, h->npblk, h->d_fx, h->d_cid, h->d_rank,
                               h->d_cell_cnt, h->ncell, lflag, h->d_err);
            ++count;
        }
        launch_scan(sc, h->d_cell_cnt, h->d_cell_start, h->ncell, a.step_dev, h->d_cur_step,
                    lflag);
    });
    run(RBE_K_SCATTER, sc, [&] {
        launch_scatter(sc, n, h->d_cid, h->d_rank, h->d_cell_start, h->d_perm_tmp, lflag,
                       h->d_err);
    });
    run(RBE_K_CELL_ORDER, sc, [&] {
        launch_order(sc, n, h->d_cid, h->d_cell_start, h->d_perm_tmp, mixed ? h->d_fx : nullptr,
                     h->d_spos, mixed ? nullptr : h->d_fx64, h->d_spos64, h->d_perm, lflag,
                     lst ? h->d_iperm : nullptr, h->d_err);
    });
    if (lst)
        run(RBE_K_LIST_BUILD, sc, [&] {
            ListArgs la{};
            la.w = make_work(h, h->d_pblk, kBlockP, 0);
            la.nblk = h->npblk;
            la.list_flag = h->d_list_flag;
            la.spos = h->d_spos;
            la.cell_start = h->d_cell_start;
            la.nbr = h->d_nbr;
            la.ncnt = h->d_ncnt;
            la.stride = std::max(h->ntot, 1);
            la.cap = h->list_cap;
            la.sref = h->d_sref;
            la.perm = h->d_perm;
            la.stats = h->d_list_stats;
            la.err = h->d_err;
            launch_list_build(sc, one, la);
        });
    if (fourier && !a.list) cudaStreamWaitEvent(st, h->ev_join, 0);
    RealArgs r = make_real_args(h, a.parts);
    r.F_out = a.F;
    r.phi_out = a.phi;
    r.md_pos = a.md_pos;
    r.md_vel = a.md_vel;
    r.F_out64 = a.F64;
    r.phi_out64 = a.phi64;
    r.md_pos64 = a.md_pos64;
    r.md_vel64 = a.md_vel64;
    r.nh = pa.nh;
    r.blk_e = a.E ? h->d_blk_e : nullptr;
    r.blk_w = (a.E && a.W) ? h->d_blk_w : nullptr;
    if (a.list) {
        r.lw = make_work(h, h->d_lblk, kBlockP / h->lsplit, 0);
        r.nlblk = h->nlblk;
        r.lsplit = h->lsplit;
        r.nbr = h->d_nbr;
        r.ncnt = h->d_ncnt;
        r.nbr_stride = std::max(h->ntot, 1);
        r.nbr_cap = h->list_cap;
        r.list_flag = h->d_list_flag;
        r.freal = h->d_freal;
        // the real-space pass over a standing list right after the prep kernel
        // (concurrent with the structure factors and the rebuild stream), or
        // over the rebuilt list at the end of the rebuild stream; then the
        // Fourier force, which adds it and applies the thermostat
        r.list_when = 0;
        if (!fused) {
            cudaStreamWaitEvent(st2, h->ev_prep, 0);
            run(RBE_K_REAL, st2, [&] { launch_real_list(st2, one, r); });
            cudaEventRecord(h->ev_real, st2);
        }
        RealArgs rb = r;
        rb.list_when = 1;
        launch_real_list(sc, one, rb);
        ++count;
        cudaEventRecord(h->ev_chain, sc);
        if (!fused) cudaStreamWaitEvent(st, h->ev_real, 0);
        cudaStreamWaitEvent(st, h->ev_chain, 0);
        MdOut md{};
        md.freal = h->d_freal;
        md.F_out = a.F;
        md.md_pos = a.md_pos;
        md.md_vel = a.md_vel;
        md.nh = pa.nh;
        md.cur_step = h->d_cur_step;
        md.list_flag = h->d_list_flag;
        if (a.done) {
            md.done_cnt = h->d_done_cnt;
            md.done_host = a.done;
            md.err_host = (int*)(a.done - 1);
            md.err = h->d_err;
        }
        run(RBE_K_FOURIER_FORCE, st, [&] { launch_force(h, st, true, md, !prof); });
    } else if (!a.list_forces) {
        run(RBE_K_REAL, st, [&] {
            if (mixed) launch_real_mixed(st, one, r); else launch_real_f64(st, one, r);
        });
    }
    if (a.list_forces) {
        // forces call: one pass over the (possibly rebuilt) list after the
        // Fourier force, assembling F, dE/dq and the energy / virial partials
        r.lw = make_work(h, h->d_lblk, kBlockP / h->lsplit, 0);
        r.nlblk = h->nlblk;
        r.lsplit = h->lsplit;
        r.nbr = h->d_nbr;
        r.ncnt = h->d_ncnt;
        r.nbr_stride = std::max(h->ntot, 1);
        r.nbr_cap = h->list_cap;
        r.list_flag = h->d_list_flag;
        r.list_when = 2;
        r.fmode = 1;
        r.flag_clear = h->d_list_flag;
        run(RBE_K_REAL, st, [&] { launch_real_list(st, one, r); });
    }
    if (a.E)
        run(RBE_K_ENERGY, st, [&] {
            launch_energy(st, one, make_work(h, nullptr, 0, 0), h->nsys, h->d_ksamp, h->d_rho_fx,
                          h->d_blk_e, h->d_blk_q, r.blk_w, a.parts,
                          a.list_forces ? 2 : (mixed ? 1 : 0), a.E,
                          r.blk_w ? a.W : nullptr);
        });
    if (prof) {
        cudaStreamSynchronize(st);                      // every branch has joined st
        for (int k = 0; k < RBE_K_COUNT; ++k) {
            if (!used[k]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, h->ev_beg[k], h->ev_end[k]) == cudaSuccess) {
                h->prof_ms[k] += ms;
                h->prof_cnt[k] += 1;
            }
        }
    }
    if (st == h->stream) h->kernel_count += count;
    return count;
}

rbe_status check_n(rbe_ctx* h, int n) {
    if (n < 0) return fail(h, RBE_ERR_ARG, "n must be >= 0");
    if (h->batch) {
        if (n != h->ntot) return fail(h, RBE_ERR_STATE, "batch handle: n must equal the total particle count");
    } else if (n > h->sys[0].p.n_max) {
        return fail(h, RBE_ERR_ARG, "n exceeds n_max");
    }
    return RBE_OK;
}

rbe_status finish(rbe_ctx* h, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, where);
    return RBE_OK;
}

// A mixed forces call on a handle that keeps a neighbour list goes over the
// list too (rebuilt when a particle moved more than skin/2); the first such
// call after anything else touched the sorted arrays builds it.
rbe_status use_list_forces(rbe_ctx* h, int n, EvalArgs& a) {
    if (!h->list || a.prec != RBE_MIXED || n <= 0) return RBE_OK;
    a.list_forces = true;
    if (!h->list_valid)
        RBE_CUDA(h, cudaMemsetAsync(h->d_list_flag, 0xFF, sizeof(int), h->stream));
    h->list_valid = true;
    return RBE_OK;
}

rbe_status forces_impl(rbe_ctx* h, int n, int prec, const void* pos, uint64_t step, int parts,
                       void* F, double* E, void* phi) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    rbe_status s = check_n(h, n);
    if (s != RBE_OK) return s;
    if (parts < 0 || parts > RBE_PART_ALL) return fail(h, RBE_ERR_ARG, "bad parts mask");
    if (n > 0 && (!pos || !F)) return fail(h, RBE_ERR_ARG, "pos_q and F_out must be non-null");
    if ((s = prepare(h, n)) != RBE_OK) return s;
    EvalArgs a{};
    a.prec = prec;
    a.parts = parts;
    a.step = step;
    a.E = E;
    if (prec == RBE_MIXED) {
        a.pos = (const float4*)pos;
        a.F = (float4*)F;
        a.phi = (float*)phi;
    } else {
        a.pos64 = (const double4*)pos;
        a.F64 = (double4*)F;
        a.phi64 = (double*)phi;
    }
    if ((s = use_list_forces(h, n, a)) != RBE_OK) return s;
    enqueue_eval(h, h->stream, a);
    return finish(h, "rbe_forces");
}

// Wave vectors of the half space {m_x > 0} u {m_x = 0, m_y > 0} u {m = (0,0,m_z>0)}
// of the cube |m|_inf <= mmax: each pair (m, -m) once.
static void half_space_cube(int mmax, std::vector<int4>& out) {
    for (int a = 0; a <= mmax; ++a)
        for (int b = -mmax; b <= mmax; ++b)
            for (int c = -mmax; c <= mmax; ++c) {
                if (a == 0 && (b < 0 || (b == 0 && c <= 0))) continue;
                out.push_back(make_int4(a, b, c, 0));
            }
}

rbe_status observables_impl(rbe_ctx* h, int n, const float* pos_q, const float* vel, int mmax,
                            double* out) {
    if (!h || !out) return fail(h, RBE_ERR_ARG, "null argument");
    rbe_status s = check_n(h, n);
    if (s != RBE_OK) return s;
    if (n > 0 && !pos_q) return fail(h, RBE_ERR_ARG, "pos_q must be non-null");
    int mm = mmax;
    if (mm <= 0)
        for (auto& sh : h->sys) mm = std::max(mm, sh.M);
    const long long side = 2LL * mm + 1;
    if ((side * side * side - 1) / 2 > (1LL << 24))
        return fail(h, RBE_ERR_ARG, "mmax too large (more than 2^24 wave vectors)");
    if ((s = prepare(h, n)) != RBE_OK) return s;
    if (h->obs_mmax != mm) {                         // wave-vector lists, once per mmax
        std::vector<int4> all, one;
        half_space_cube(mm, one);
        h->obs_off.assign(h->nsys, 0);
        h->obs_K.assign(h->nsys, (int)one.size());
        for (int sy = 0; sy < h->nsys; ++sy) {
            h->obs_off[sy] = (int)all.size();
            all.insert(all.end(), one.begin(), one.end());
        }
        if (h->d_obs_m) cudaFree(h->d_obs_m);
        if (h->d_obs_rho) cudaFree(h->d_obs_rho);
        if (h->d_obs_part) cudaFree(h->d_obs_part);
        h->d_obs_m = nullptr;
        h->d_obs_rho = nullptr;
        h->d_obs_part = nullptr;
        if (dalloc(&h->d_obs_m, all.size()) != RBE_OK ||
            dalloc(&h->d_obs_rho, 2 * all.size()) != RBE_OK ||
            dalloc(&h->d_obs_part, (one.size() + 255) / 256 + 1) != RBE_OK ||
            (!h->d_obs_w && dalloc(&h->d_obs_w, 2 * (size_t)h->nsys) != RBE_OK) ||
            (!h->d_obs_out && dalloc(&h->d_obs_out, 12 * (size_t)h->nsys) != RBE_OK))
            return fail(h, RBE_ERR_OOM, "cudaMalloc failed: observables workspace");
        RBE_CUDA(h, cudaMemcpy(h->d_obs_m, all.data(), sizeof(int4) * all.size(),
                               cudaMemcpyHostToDevice));
        h->obs_mmax = mm;
    }
    // real-space Coulomb and LJ energies and virials (mixed path), fixed-point positions
    EvalArgs a{};
    a.prec = RBE_MIXED;
    a.parts = RBE_PART_REAL | RBE_PART_LJ;
    a.pos = (const float4*)pos_q;
    a.E = h->d_stage_E;
    a.W = h->d_obs_w;
    if ((s = use_list_forces(h, n, a)) != RBE_OK) return s;
    enqueue_eval(h, h->stream, a);
    for (int sy = 0; sy < h->nsys; ++sy) {
        const SysHost& sh = h->sys[sy];
        launch_observables(h->stream, h->sysdev[sy], h->d_fx, sh.off_p, sh.n,
                           h->d_obs_m + h->obs_off[sy], h->obs_K[sy],
                           h->d_obs_rho + 2 * (size_t)h->obs_off[sy], h->d_obs_part,
                           (const float4*)pos_q,
                           (const float4*)vel, h->d_stage_E + 4 * sy, h->d_obs_w + 2 * sy,
                           sh.p.mass, h->d_obs_out + 12 * sy);
    }
    RBE_CUDA(h, cudaMemcpyAsync(out, h->d_obs_out, sizeof(double) * 12 * h->nsys,
                                cudaMemcpyDeviceToHost, h->stream));
    RBE_CUDA(h, cudaStreamSynchronize(h->stream));
    return finish(h, "rbe_observables");
}

// The device address of page-locked host memory (its own address under
// unified addressing), or null for pageable memory.
void* mapped_host(void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();                       // pageable memory on some drivers
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// A host-buffer step (rbe_step_host): the caller's arrays copied into the
// staging buffers before the steps and back after them, the step index from
// the pinned word, the device error word back into the pinned word.
struct HostIO {
    float* pos;
    float* vel;
};

rbe_status step_impl(rbe_ctx* h, int n, int prec, void* pos, void* vel, int nsteps,
                     uint64_t* step_dev, float* F_out = nullptr, const HostIO* io = nullptr,
                     unsigned long long* done = nullptr) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    rbe_status s = check_n(h, n);
    if (s != RBE_OK) return s;
    if (nsteps < 0) return fail(h, RBE_ERR_ARG, "nsteps must be >= 0");
    if (!step_dev) return fail(h, RBE_ERR_ARG, "step_dev must be non-null");
    if (n > 0 && (!pos || !vel)) return fail(h, RBE_ERR_ARG, "pos_q and vel must be non-null");
    if ((s = prepare(h, n)) != RBE_OK) return s;
    EvalArgs a{};
    a.prec = prec;
    a.parts = RBE_PART_ALL;
    a.step_dev = step_dev;
    if (prec == RBE_MIXED) {
        a.pos = (const float4*)pos;
        a.md_pos = (float4*)pos;
        a.md_vel = (float4*)vel;
        a.F = (float4*)F_out;
        a.list = h->list;
        a.done = h->list ? done : nullptr;
    } else {
        a.pos64 = (const double4*)pos;
        a.md_pos64 = (double4*)pos;
        a.md_vel64 = (double4*)vel;
    }
    if (a.list) {
        // the first step after anything else touched the sorted arrays builds a list
        if (!h->list_valid && nsteps > 0)
            RBE_CUDA(h, cudaMemsetAsync(h->d_list_flag, 0xFF, sizeof(int), h->stream));
        if (nsteps > 0) h->list_valid = true;
    } else if (nsteps > 0) {
        h->list_valid = false;
    }
    const size_t bytes = sizeof(float4) * (size_t)n;
    // the copies of a host-buffer call, on stream sq
    auto copy_in = [&](cudaStream_t sq) {
        if (n > 0) {
            cudaMemcpyAsync(pos, io->pos, bytes, cudaMemcpyHostToDevice, sq);
            cudaMemcpyAsync(vel, io->vel, bytes, cudaMemcpyHostToDevice, sq);
        }
        cudaMemcpyAsync(step_dev, h->h_pin, sizeof(uint64_t), cudaMemcpyHostToDevice, sq);
    };
    auto copy_out = [&](cudaStream_t sq) {
        if (n > 0) {
            cudaMemcpyAsync(io->pos, pos, bytes, cudaMemcpyDeviceToHost, sq);
            cudaMemcpyAsync(io->vel, vel, bytes, cudaMemcpyDeviceToHost, sq);
        }
        cudaMemcpyAsync(h->h_pin + 1, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, sq);
    };
    // a host-buffer call replays one graph holding copies and steps (up to 4)
    const bool host_graph = io && nsteps <= 4;
    if (!h->use_graph || h->prof_on) {
        if (io) copy_in(h->stream);
        for (int k = 0; k < nsteps; ++k) enqueue_eval(h, h->stream, a);
        if (io) copy_out(h->stream);
        return finish(h, "rbe_step");
    }
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    for (auto& g : h->graphs)
        if (g.n == n && g.pos == pos && g.vel == vel && g.step == step_dev && g.prec == prec &&
            g.F == (const void*)F_out && g.host_pos == (host_graph ? io->pos : nullptr) &&
            g.host_vel == (host_graph ? io->vel : nullptr) &&
            g.host_steps == (host_graph ? nsteps : 0) && g.done == (const void*)a.done) {
            exec = g.exec;
            kernels = g.kernels;
        }
    if (!exec) {
        // Capture on the handle's private stream, then replay on the caller's.
        RBE_CUDA(h, cudaStreamSynchronize(h->stream));
        RBE_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        if (host_graph) {
            copy_in(h->cap_stream);
            kernels = 0;
            for (int k = 0; k < nsteps; ++k) kernels += enqueue_eval(h, h->cap_stream, a);
            copy_out(h->cap_stream);
        } else {
            kernels = enqueue_eval(h, h->cap_stream, a);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        h->graphs.push_back(GraphEntry{n, pos, vel, step_dev, F_out, prec,
                                       host_graph ? io->pos : nullptr,
                                       host_graph ? io->vel : nullptr,
                                       host_graph ? nsteps : 0, a.done, exec, kernels});
    }
    if (host_graph) {
        RBE_CUDA(h, cudaGraphLaunch(exec, h->stream));
        h->kernel_count += kernels;
    } else {
        if (io) copy_in(h->stream);
        for (int k = 0; k < nsteps; ++k) RBE_CUDA(h, cudaGraphLaunch(exec, h->stream));
        if (io) copy_out(h->stream);
        h->kernel_count += (int64_t)kernels * nsteps;
    }
    return finish(h, "rbe_step");
}

}  // namespace

namespace {
// Device time of `reps` launches of one kernel (the first, a warm-up, dropped).
template <class F>
float time_kernel(rbe_ctx* h, cudaEvent_t e0, cudaEvent_t e1, F&& launch) {
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, h->stream);
        launch();
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;
    }
    return tot;
}
}  // namespace

namespace {
// Wait until h's stream has finished its queued work.  Without a wait limit
// this is cudaStreamSynchronize; with one (rbe_set_wait_limit) the stream is
// polled until it is idle or the limit has passed, and then the call returns
// RBE_ERR_TIMEOUT with the work still queued.
rbe_status wait_stream(rbe_ctx* h, const char* where) {
    if (!(h->wait_limit > 0.0)) {
        RBE_CUDA(h, cudaStreamSynchronize(h->stream));
        return RBE_OK;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(h->stream);
        if (e == cudaSuccess) return RBE_OK;
        if (e != cudaErrorNotReady) return cuda_fail(h, e, where);
        const double dt =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > h->wait_limit) return timeout_fail(h);
        std::this_thread::yield();
    }
}

// The device error word as read back into the pinned word (after a
// synchronisation): latched conditions become a status, and the word is cleared.
rbe_status report_err(rbe_ctx* h) {
    int err = 0;
    std::memcpy(&err, h->h_pin + 1, sizeof(int));
    if (err) {
        RBE_CUDA(h, cudaMemset(h->d_err, 0, sizeof(int)));
        if (err & kErrSampler)
            return fail(h, RBE_ERR_SAMPLER, "a k-sample drew (0,0,0) on 32 attempts in a row");
        if (err & kErrList)
            return fail(h, RBE_ERR_LIST, "a particle had more neighbours within r_c + skin than "
                                         "the list holds (" + std::to_string(h->list_cap) + ")");
        if (err & kErrNonfinite)
            return fail(h, RBE_ERR_NONFINITE, "a position or charge of the input was NaN or "
                                              "infinite (the results of those calls are not "
                                              "meaningful)");
        if (err & kErrBounds)
            return fail(h, RBE_ERR_BOUNDS, "the bounds-checked build found an index outside its "
                                           "array (the access was skipped)");
    }
    return finish(h, "rbe_sync");
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

rbe_status rbe_create(const rbe_params* p, rbe_handle* out) {
    if (!p) return fail(nullptr, RBE_ERR_ARG, "params is NULL");
    return create_common(p, nullptr, 1, false, out);
}

rbe_status rbe_create_batch(const rbe_params* per_replica, const int32_t* n_per_replica,
                            int32_t n_replicas, rbe_handle* out) {
    if (!per_replica || !n_per_replica || n_replicas < 1)
        return fail(nullptr, RBE_ERR_ARG, "bad batch arguments");
    return create_common(per_replica, n_per_replica, n_replicas, true, out);
}

void rbe_destroy(rbe_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    release(h);
    delete h;
}

const char* rbe_last_error(rbe_handle h) {
    if (h) return h->err.c_str();
    return g_last_error.c_str();
}

rbe_status rbe_set_stream(rbe_handle h, void* cuda_stream) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    h->stream = (cudaStream_t)cuda_stream;
    return RBE_OK;
}

rbe_status rbe_get_info(rbe_handle h, int32_t sys, rbe_info* info) {
    if (!h || !info) return fail(h, RBE_ERR_ARG, "null argument");
    if (sys < 0 || sys >= h->nsys) return fail(h, RBE_ERR_ARG, "system index out of range");
    const SysHost& s = h->sys[sys];
    std::memset(info, 0, sizeof(*info));
    info->H = s.H;
    info->S = s.S;
    info->M = s.M;
    info->n_cells_dim = s.ncd;
    info->n = h->batch ? s.n : s.p.n_max;
    info->P = s.p.P;
    info->n_systems = h->nsys;
    info->first_particle = s.off_p;
    info->first_k = s.off_k;
    return RBE_OK;
}

rbe_status rbe_get_table(rbe_handle h, int32_t sys, uint64_t* table_out) {
    if (!h || !table_out) return fail(h, RBE_ERR_ARG, "null argument");
    if (sys < 0 || sys >= h->nsys) return fail(h, RBE_ERR_ARG, "system index out of range");
    std::memcpy(table_out, h->sys[sys].table.data(), sizeof(uint64_t) * h->sys[sys].table.size());
    return RBE_OK;
}

rbe_status rbe_sample_k(rbe_handle h, uint64_t step, int32_t* m_out) {
    if (!h || !m_out) return fail(h, RBE_ERR_ARG, "null argument");
    const int n = h->batch ? h->ntot : std::max(h->cur_n, 0);
    rbe_status s = prepare(h, n);
    if (s != RBE_OK) return s;
    if (h->mh) {
        // the chains are consumed in order: report the batch of the last evaluation
        RBE_CUDA(h, cudaMemcpyAsync(m_out, h->d_ksamp, sizeof(int4) * h->ktot,
                                    cudaMemcpyDeviceToDevice, h->stream));
    } else {
        RBE_CUDA(h, cudaMemcpyAsync(h->d_stage_step, &step, sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, h->stream));
        launch_sample(h->stream, h->d_sys, h->nsys, h->ktot, h->d_kstart, h->d_table,
                      h->d_stage_step, (int4*)m_out, h->d_err);
    }
    RBE_CUDA(h, cudaStreamSynchronize(h->stream));
    return finish(h, "rbe_sample_k");
}

rbe_status rbe_observables(rbe_handle h, int32_t n, const float* pos_q, const float* vel,
                           int32_t mmax, double* out) {
    return observables_impl(h, n, pos_q, vel, mmax, out);
}

rbe_status rbe_forces(rbe_handle h, int32_t n, const float* pos_q, uint64_t step, float* F_out,
                      double* E_out, float* phi_out) {
    return forces_impl(h, n, RBE_MIXED, pos_q, step, RBE_PART_ALL, F_out, E_out, phi_out);
}

rbe_status rbe_forces_ex(rbe_handle h, int32_t n, const float* pos_q, uint64_t step,
                         int32_t parts, float* F_out, double* E_out, float* phi_out) {
    return forces_impl(h, n, RBE_MIXED, pos_q, step, parts, F_out, E_out, phi_out);
}

rbe_status rbe_forces_f64(rbe_handle h, int32_t n, const double* pos_q, uint64_t step,
                          int32_t parts, double* F_out, double* E_out, double* phi_out) {
    return forces_impl(h, n, RBE_FP64, pos_q, step, parts, F_out, E_out, phi_out);
}

rbe_status rbe_step(rbe_handle h, int32_t n, float* pos_q, float* vel, int32_t nsteps,
                    uint64_t* step_dev) {
    return step_impl(h, n, RBE_MIXED, pos_q, vel, nsteps, step_dev);
}

rbe_status rbe_step_f64(rbe_handle h, int32_t n, double* pos_q, double* vel, int32_t nsteps,
                        uint64_t* step_dev) {
    return step_impl(h, n, RBE_FP64, pos_q, vel, nsteps, step_dev);
}

rbe_status rbe_step_ex(rbe_handle h, int32_t n, float* pos_q, float* vel, int32_t nsteps,
                       uint64_t* step_dev, float* F_out) {
    return step_impl(h, n, RBE_MIXED, pos_q, vel, nsteps, step_dev, F_out);
}

rbe_status rbe_list_stats(rbe_handle h, int64_t* builds, int32_t* max_count, int32_t* capacity) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    unsigned long long st[2] = {0ull, 0ull};
    if (h->list) {
        RBE_CUDA(h, cudaStreamSynchronize(h->stream));
        RBE_CUDA(h, cudaMemcpy(st, h->d_list_stats, sizeof(st), cudaMemcpyDeviceToHost));
    }
    if (builds) *builds = (int64_t)st[0];
    if (max_count) *max_count = (int32_t)st[1];
    if (capacity) *capacity = h->list ? h->list_cap : 0;
    return finish(h, "rbe_list_stats");
}

rbe_status rbe_nose_hoover_xi(rbe_handle h, double* xi, int32_t set) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    if (!xi) return fail(h, RBE_ERR_ARG, "xi is NULL");
    std::vector<NhState> nh(h->nsys);
    if (set) {
        for (int sy = 0; sy < h->nsys; ++sy) {
            nh[sy] = NhState{};
            nh[sy].xi = xi[sy];
            nh[sy].first = 1;
        }
        RBE_CUDA(h, cudaMemcpyAsync(h->d_nh, nh.data(), sizeof(NhState) * h->nsys,
                                    cudaMemcpyHostToDevice, h->stream));
        RBE_CUDA(h, cudaStreamSynchronize(h->stream));
    } else {
        RBE_CUDA(h, cudaMemcpyAsync(nh.data(), h->d_nh, sizeof(NhState) * h->nsys,
                                    cudaMemcpyDeviceToHost, h->stream));
        RBE_CUDA(h, cudaStreamSynchronize(h->stream));
        for (int sy = 0; sy < h->nsys; ++sy) xi[sy] = nh[sy].xi;
    }
    return finish(h, "rbe_nose_hoover_xi");
}

rbe_status rbe_set_graph(rbe_handle h, int32_t use_graph) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    h->use_graph = use_graph != 0;
    return RBE_OK;
}

rbe_status rbe_forces_host(rbe_handle h, int32_t n, const float* pos_q, uint64_t step,
                           float* F_out, double* E_out) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    rbe_status s = check_n(h, n);
    if (s != RBE_OK) return s;
    if (n > 0 && (!pos_q || !F_out)) return fail(h, RBE_ERR_ARG, "null host buffer");
    const size_t bytes = sizeof(float4) * (size_t)n;
    if (n > 0)
        RBE_CUDA(h, cudaMemcpyAsync(h->d_stage_pos, pos_q, bytes, cudaMemcpyHostToDevice, h->stream));
    s = forces_impl(h, n, RBE_MIXED, h->d_stage_pos, step, RBE_PART_ALL, h->d_stage_F,
                    E_out ? h->d_stage_E : nullptr, nullptr);
    if (s != RBE_OK) return s;
    if (n > 0)
        RBE_CUDA(h, cudaMemcpyAsync(F_out, h->d_stage_F, bytes, cudaMemcpyDeviceToHost, h->stream));
    if (E_out)
        RBE_CUDA(h, cudaMemcpyAsync(E_out, h->d_stage_E, sizeof(double) * 4 * h->nsys,
                                    cudaMemcpyDeviceToHost, h->stream));
    return rbe_sync(h);
}

rbe_status rbe_step_host(rbe_handle h, int32_t n, float* pos_q, float* vel, int32_t nsteps,
                         uint64_t step0) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    rbe_status s = check_n(h, n);
    if (s != RBE_OK) return s;
    if (n > 0 && (!pos_q || !vel)) return fail(h, RBE_ERR_ARG, "null host buffer");
    h->h_pin[0] = step0;
    void* dpos = n > 0 ? mapped_host(pos_q) : nullptr;
    void* dvel = n > 0 ? mapped_host(vel) : nullptr;
    if (n > 0 && dpos && dvel) {
        // page-locked arrays: the step's kernels read and write them in place
        // over the host link (no staging copies); the step index advances in
        // the pinned word.  A list step's closing kernel also delivers the
        // error word and then a completion word there, which this thread
        // polls instead of waiting on the stream.
        const bool signal = h->list && nsteps > 0;
        const uint64_t want = step0 + (uint64_t)nsteps;
        uint64_t* done = h->h_pin + 2;
        if (signal) __atomic_store_n(done, ~want, __ATOMIC_RELAXED);
        s = step_impl(h, n, RBE_MIXED, dpos, dvel, nsteps, h->h_pin_dev, nullptr, nullptr,
                      signal ? (unsigned long long*)(h->h_pin_dev + 2) : nullptr);
        if (s != RBE_OK) return s;
        if (signal) {
            // acquire: the outputs and the error word, stored before the word
            // on the device side, are read after it here
            bool seen = false;
            const bool limited = h->wait_limit > 0.0;
            const auto t0 = std::chrono::steady_clock::now();
            for (unsigned it = 1; !(seen = __atomic_load_n(done, __ATOMIC_ACQUIRE) == want); ++it) {
                if ((it & 1023u) == 0 && cudaStreamQuery(h->stream) != cudaErrorNotReady) break;
                if (limited && (it & 63u) == 0 &&
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
                        h->wait_limit)
                    return timeout_fail(h);
            }
            if (seen || __atomic_load_n(done, __ATOMIC_ACQUIRE) == want) return report_err(h);
            // the stream ended without the signal: its status decides
        }
        RBE_CUDA(h, cudaMemcpyAsync(h->h_pin + 1, h->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                    h->stream));
    } else {
        const HostIO io{pos_q, vel};          // pageable: staged through device buffers
        s = step_impl(h, n, RBE_MIXED, h->d_stage_pos, h->d_stage_vel, nsteps, h->d_stage_step,
                      nullptr, &io);
        if (s != RBE_OK) return s;
    }
    // the outputs and the error word are queued: one synchronisation
    if ((s = wait_stream(h, "rbe_step_host")) != RBE_OK) return s;
    return report_err(h);
}

rbe_status rbe_sync(rbe_handle h) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    // the error word follows the queued work in the stream: one synchronisation
    RBE_CUDA(h, cudaMemcpyAsync(h->h_pin + 1, h->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                h->stream));
    const rbe_status s = wait_stream(h, "rbe_sync");
    if (s != RBE_OK) return s;
    return report_err(h);
}

rbe_status rbe_set_wait_limit(rbe_handle h, double seconds) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    if (!(seconds >= 0.0) || !std::isfinite(seconds))
        return fail(h, RBE_ERR_ARG, "the wait limit must be a finite number of seconds >= 0");
    h->wait_limit = seconds;
    return RBE_OK;
}

rbe_status rbe_set_fusion(rbe_handle h, int32_t on) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    if (on != -1 && on != 0 && on != 1)
        return fail(h, RBE_ERR_ARG, "fusion must be -1 (automatic), 0 or 1");
    h->fusion_mode = on;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return RBE_OK;
}

rbe_status rbe_get_fusion(rbe_handle h, int32_t* on) {
    if (!h || !on) return fail(h, RBE_ERR_ARG, "null argument");
    *on = fusion_on(h) ? 1 : 0;
    return RBE_OK;
}

rbe_status rbe_set_tuning(rbe_handle h, const rbe_tuning* t) {
    if (!h || !t) return fail(h, RBE_ERR_ARG, "null argument");
    const int c = t->rho_chunk, f = t->force_split, r = t->real_split, sg = t->real_seg;
    if (c != 0 && (c < 32 || c > 8192 || (c & (c - 1))))
        return fail(h, RBE_ERR_ARG, "rho_chunk must be 0 or a power of two in [32, 8192]");
    if (f != 0 && f != 1 && f != 2 && f != 4 && f != 8)
        return fail(h, RBE_ERR_ARG, "force_split must be 0, 1, 2, 4 or 8");
    if (r != 0 && r != 1 && r != 3 && r != 9)
        return fail(h, RBE_ERR_ARG, "real_split must be 0, 1, 3 or 9");
    if (sg < 0 || sg > 256) return fail(h, RBE_ERR_ARG, "real_seg must be in [0, 256]");
    const int ls = t->list_split;
    if (ls != 0 && ls != 1 && ls != 2 && ls != 4 && ls != 8)
        return fail(h, RBE_ERR_ARG, "list_split must be 0, 1, 2, 4 or 8");
    h->list_split = ls;
    h->rho_chunk = c;
    h->force_split = f;
    h->real_split = r;
    h->real_seg = sg;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return RBE_OK;
}

rbe_status rbe_get_tuning(rbe_handle h, rbe_tuning* t) {
    if (!h || !t) return fail(h, RBE_ERR_ARG, "null argument");
    const long long ntot = h->batch ? h->ntot : std::max(h->cur_n, 0);
    t->rho_chunk = h->cur_chunk > 0 ? h->cur_chunk
                                    : (h->rho_chunk > 0 ? h->rho_chunk : auto_chunk(h, ntot));
    t->force_split = h->cur_split > 0 ? h->cur_split
                                      : (h->force_split > 0 ? h->force_split : auto_split(ntot));
    t->real_split = h->cur_rsplit > 0 ? h->cur_rsplit
                                      : (h->real_split > 0 ? h->real_split
                                                           : auto_real_split(ntot));
    int ncd_max = 3;
    for (auto& sh : h->sys) ncd_max = std::max(ncd_max, sh.ncd);
    t->real_seg = h->cur_seg > 0 ? h->cur_seg
                                 : (h->real_seg > 0 ? std::min(h->real_seg, ncd_max)
                                                    : auto_real_seg(ntot, h->ncell, ncd_max));
    t->list_split = h->cur_lsplit > 0 ? h->cur_lsplit
                                      : (h->list_split > 0 ? h->list_split : auto_list_split(ntot));
    return RBE_OK;
}


rbe_status rbe_autotune(rbe_handle h, int32_t n, const float* pos_q, rbe_tuning* out) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    rbe_status s = check_n(h, n);
    if (s != RBE_OK) return s;
    if (n > 0 && !pos_q) return fail(h, RBE_ERR_ARG, "pos_q is NULL");
    cudaEvent_t e0, e1;
    RBE_CUDA(h, cudaEventCreate(&e0));
    RBE_CUDA(h, cudaEventCreate(&e1));
    EvalArgs a{};
    a.prec = RBE_MIXED;
    a.parts = RBE_PART_ALL;
    a.pos = (const float4*)pos_q;
    a.F = h->d_stage_F;
    const bool prof = h->prof_on;
    h->prof_on = false;
    // structure-factor chunk
    float best = 1e30f;
    int best_chunk = 32;
    for (int c = 32; c <= 4096; c <<= 1) {
        h->rho_chunk = c;
        if ((s = prepare(h, n)) != RBE_OK) break;
        enqueue_eval(h, h->stream, a);
        const float t = time_kernel(h, e0, e1, [&] { launch_rho(h, h->stream, true); });
        if (t < best) { best = t; best_chunk = c; }
    }
    h->rho_chunk = best_chunk;
    // Fourier-force split, timed in the form the handle's MD steps run it
    // (with a neighbour list: the step variant, which adds the real-space
    // force and takes one sine per pair; without: the forces variant)
    best = 1e30f;
    int best_split = 1;
    for (int sp = 1; sp <= 8 && s == RBE_OK; sp <<= 1) {
        h->force_split = sp;
        if ((s = prepare(h, n)) != RBE_OK) break;
        enqueue_eval(h, h->stream, a);
        MdOut md{};
        if (h->list) {
            md.freal = h->d_freal;            // contents irrelevant: only timed
            md.F_out = h->d_stage_F;
            md.cur_step = h->d_cur_step;
        }
        const float t = time_kernel(h, e0, e1, [&] { launch_force(h, h->stream, true, md); });
        if (t < best) { best = t; best_split = sp; }
    }
    h->force_split = best_split;
    // real-space segment length and split
    best = 1e30f;
    int best_rsplit = 1, best_seg = 1;
    int ncd_max = 3;
    for (auto& sh : h->sys) ncd_max = std::max(ncd_max, sh.ncd);
    std::vector<int> segs_try;
    for (int sg = 1; sg <= ncd_max; sg = sg < 4 ? sg + 1 : sg * 2) segs_try.push_back(sg);
    if (segs_try.back() != ncd_max) segs_try.push_back(ncd_max);
    for (int sg : segs_try) {
        for (int sp = 1; sp <= 9 && s == RBE_OK; sp *= 3) {
            h->real_split = sp;
            h->real_seg = sg;
            if ((s = prepare(h, n)) != RBE_OK) break;
            if ((long long)h->nseg * 2 < 152 && sg > 1) continue;   // too few blocks
            enqueue_eval(h, h->stream, a);
            RealArgs r = make_real_args(h, RBE_PART_ALL);
            r.F_out = h->d_stage_F;
            const float t = time_kernel(h, e0, e1, [&] { launch_real_mixed(h->stream, !h->batch, r); });
            if (t < best) { best = t; best_rsplit = sp; best_seg = sg; }
        }
    }
    h->real_split = best_rsplit;
    h->real_seg = best_seg;
    // neighbour-list pass: lanes per particle, timed on a list built for this
    // input.  Fused, it is timed inside the launch it shares with the
    // structure factors, and the structure-factor chunk is re-chosen with it
    // (the shapes fastest alone are not always the fastest together).  With
    // fusion automatic both forms are tuned, a whole list evaluation is timed
    // in each, and the faster is kept.
    int best_lsplit = 0;
    if (h->list) {
        const int mode = h->fusion_mode;
        const int rho_best_chunk = best_chunk;
        auto build_list = [&](EvalArgs& b) -> rbe_status {
            rbe_status st = prepare(h, n);
            if (st != RBE_OK) return st;
            b = a;
            b.list = true;
            RBE_CUDA(h, cudaMemsetAsync(h->d_list_flag, 0xFF, sizeof(int), h->stream));
            enqueue_eval(h, h->stream, b);
            return RBE_OK;
        };
        // the list split (and, fused, the chunk) of one form: its best kernel time
        auto tune_form = [&](bool fused, int& out_chunk, int& out_ls) {
            h->fusion_mode = fused ? 1 : 0;
            std::vector<int> chunks{rho_best_chunk};
            if (fused) {
                if (rho_best_chunk / 2 >= 32) chunks.insert(chunks.begin(), rho_best_chunk / 2);
                if (rho_best_chunk * 2 <= 4096) chunks.push_back(rho_best_chunk * 2);
            }
            float bt = 1e30f;
            out_chunk = rho_best_chunk;
            out_ls = 1;
            for (int c : chunks) {
                h->rho_chunk = c;
                for (int ls = 1; ls <= 8 && s == RBE_OK; ls <<= 1) {
                    h->list_split = ls;
                    EvalArgs b{};
                    if ((s = build_list(b)) != RBE_OK) break;
                    RealArgs r = make_real_args(h, RBE_PART_ALL);
                    r.F_out = h->d_stage_F;
                    r.lw = make_work(h, h->d_lblk, kBlockP / h->lsplit, 0);
                    r.nlblk = h->nlblk;
                    r.lsplit = h->lsplit;
                    r.nbr = h->d_nbr;
                    r.ncnt = h->d_ncnt;
                    r.nbr_stride = std::max(h->ntot, 1);
                    r.nbr_cap = h->list_cap;
                    r.list_flag = h->d_list_flag;
                    r.list_when = 0;
                    r.freal = h->d_freal;
                    const int ltiles = (h->pmax + kRhoKT - 1) / kRhoKT;
                    const float t = time_kernel(h, e0, e1, [&] {
                        if (fused)
                            launch_rho_list(h->stream, !h->batch,
                                            make_work(h, h->d_chunks, h->cur_chunk, 1),
                                            h->nchunks, ltiles, h->d_ksamp, h->d_kcoef, h->d_fx,
                                            h->d_rho_fx, h->d_kcnt, h->d_kab, r, false);
                        else
                            launch_real_list(h->stream, !h->batch, r);
                    });
                    if (t < bt) { bt = t; out_chunk = c; out_ls = ls; }
                }
            }
        };
        // a whole evaluation over the standing list in one form and shape
        auto time_form = [&](bool fused, int chunk, int ls) -> float {
            h->fusion_mode = fused ? 1 : 0;
            h->rho_chunk = chunk;
            h->list_split = ls;
            EvalArgs b{};
            if ((s = build_list(b)) != RBE_OK) return 1e30f;
            return time_kernel(h, e0, e1, [&] { enqueue_eval(h, h->stream, b); });
        };
        int fc = rho_best_chunk, fls = 1, sc = rho_best_chunk, sls = 1;
        float tf = 1e30f, ts = 1e30f;
        if (mode != 0 && s == RBE_OK) {
            tune_form(true, fc, fls);
            if (s == RBE_OK) tf = time_form(true, fc, fls);
        }
        if (mode != 1 && s == RBE_OK) {
            tune_form(false, sc, sls);
            if (s == RBE_OK) ts = time_form(false, sc, sls);
        }
        const bool fuse = mode == 1 || (mode == -1 && tf < ts);
        h->fusion_mode = mode;
        if (mode == -1) h->fuse_tuned = fuse ? 1 : 0;
        best_chunk = fuse ? fc : sc;
        best_lsplit = fuse ? fls : sls;
        h->rho_chunk = best_chunk;
        h->list_split = best_lsplit;
        h->list_valid = false;
    }
    h->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != RBE_OK) return s;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    if ((s = prepare(h, n)) != RBE_OK) return s;
    if (out) {
        out->rho_chunk = best_chunk;
        out->force_split = best_split;
        out->real_split = best_rsplit;
        out->real_seg = best_seg;
        out->list_split = best_lsplit;
    }
    return finish(h, "rbe_autotune");
}

rbe_status rbe_profile(rbe_handle h, int32_t enable) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    if (enable && !h->ev_beg[0]) {
        for (int k = 0; k < RBE_K_COUNT; ++k) {
            RBE_CUDA(h, cudaEventCreate(&h->ev_beg[k]));
            RBE_CUDA(h, cudaEventCreate(&h->ev_end[k]));
        }
    }
    h->prof_on = enable != 0;
    return RBE_OK;
}

rbe_status rbe_profile_read(rbe_handle h, double* ms, int64_t* launches) {
    if (!h) return fail(nullptr, RBE_ERR_ARG, "null handle");
    for (int k = 0; k < RBE_K_COUNT; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->prof_cnt[k];
        h->prof_ms[k] = 0.0;
        h->prof_cnt[k] = 0;
    }
    return RBE_OK;
}

rbe_status rbe_launch_count(rbe_handle h, int64_t* count) {
    if (!h || !count) return fail(h, RBE_ERR_ARG, "null argument");
    *count = h->kernel_count;
    return RBE_OK;
}

}  // extern "C"

namespace rbe {
// Lets other translation units of the library report a message through
// rbe_last_error(NULL).
void set_last_error_message(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace rbe
