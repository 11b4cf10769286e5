// rbe_internal.cuh -- device-side data layout and kernel launchers of librbe.
//
// One handle holds one or more independent periodic systems ("replicas").
// Every kernel covers all systems of the handle in one launch; work items are
// (system, tile) pairs from small tables built on the host, so a single system
// is just the one-entry case of the batch.
//
// HBM layout (per handle, sized at create for the total particle count N):
//   fx     uint4 [N]   unsorted 32-bit fixed-point fractional coordinates
//                      (x/L, y/L, z/L mod 1, scaled by 2^32) and the charge bits
//   cid    int   [N]   global cell index;   rank int [N]: atomic slot within the cell
//   perm_tmp int [N]   caller's index at its atomic slot (arbitrary in-cell order)
//   spos   uint4 [N]   fx sorted by cell, in-cell by caller's index (the order all
//                      later kernels use)
//   perm   int   [N]   sorted index -> caller's index
//   fs     float4[N]   Fourier force (xyz) and Fourier dE/dq (w), caller's order
//   cell_cnt / cell_start  int [C + 1] over all systems' cells
//   rho_fx int64 [2K]  rho(k_l) = (Re, Im) accumulated over all chunks with 64-bit
//                      fixed-point atomics (integer addition is associative, so
//                      the sum is bitwise reproducible), K = sum_s P_s
//   ksamp  int4   [K] (m_x, m_y, m_z, attempts)
//   qsum_fx int64 [nsys] sum q in fixed point (for dE/dq)
//   blk_e  double2[nblk] per-block (E_coul, E_lj); blk_q double2[nblk] (sum q, sum q^2)
// and the same with double4 / double2 records for the FP64 path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rbe.h"

namespace rbe {

constexpr int kBlockP = 128;      // particles per block of the per-particle kernels
constexpr int kLTile = 128;       // threads per wave-vector row of the structure-factor kernels
constexpr int kRhoK = 2;          // wave vectors per thread of the mixed structure factors
constexpr int kRhoKT = kLTile * kRhoK;   // wave vectors per tile of the mixed structure factors
constexpr int kMaxAttempts = 32;  // bound on the (0,0,0) rejection loop
constexpr int kErrSampler = 1;    // bits in the device error word
constexpr int kErrList = 2;       // a neighbour list overflowed
constexpr int kErrNonfinite = 4;  // a position or charge of the input was NaN or infinite
constexpr int kErrBounds = 8;     // (bounds-checked build) an index fell outside its array
constexpr double kQScale = 4294967296.0;           // 2^32: fixed point of sum q

// Per-system constants (device copy).  All derived in FP64 on the host.
struct SysDev {
    double L, invL, V, alpha, sqrt_alpha, r_c, lB, S;
    double coef_scale;      // lB * (S / P) * 4 pi / V ; coef_l = coef_scale / k_l^2
    double self_coef;       // lB * sqrt(alpha / pi)
    double bg_coef;         // lB * pi / (V alpha)
    double lj_eps, lj_sigma2, lj_rcut2, lj_shift;
    double c1, c2, dt, dt_over_m;
    float fx_hi, fx_lo;     // 2^32 / L as an unevaluated float pair (hi + lo)
    float Lf, L_over_2_32;  // L and L / 2^32 in FP32
    uint64_t seed;
    uint32_t stream;
    int n, P, M, ncd;
    int off_p;              // first particle (concatenated arrays)
    int off_c;              // first cell
    int off_k;              // first k sample
    int off_t;              // first table entry
    int off_part;           // first partial of the structure-factor chunks
    int nchunk;             // structure-factor chunks of this system
    double rho_scale;       // 64-bit fixed-point scale of the rho(k) accumulators
    double rho_inv_scale;
    int off_b, nb;          // first per-particle block and block count (prep)
    int off_rb, nrb;        // first real-space block and block count (FP64 path)
    int off_sg, nsg;        // first real-space segment and segment count (mixed path)
    int off_lb, nlb;        // first neighbour-list block and block count
    // FP32 copies of the pair and Langevin constants, rounded once on the host
    // (kernels then hold no double-to-float conversions)
    float f_rc2, f_lj_rc2, f_alpha, f_sqrt_alpha, f_two_sa_spi, f_lB;
    float f_lj_sigma2, f_lj_eps, f_lj_shift;
    float f_c1, f_c2, f_dt, f_dt_over_m, f_invL;
    float f_inv_Lu;         // 2^32 / L: length to fixed-point units
    int thermostat;         // RBE_THERMO_LANGEVIN, _ANDERSEN or _NOSE_HOOVER
    uint64_t andersen_thr;  // collision iff 32-bit Philox word < nu dt 2^32
    double vsd;             // sqrt(kT / m): Andersen velocity standard deviation
    float f_vsd;
    uint32_t corner_q, corner_r;   // 2^32 = corner_q * ncd + corner_r (cell corners)
    double nh_rate;         // Nose-Hoover: dt / (3 n tau^2), xi += nh_rate (K2 / kT - 3 n)
    double nh_k2scale;      // m / kT * 2^32: fixed-point units of the kinetic sum
    // neighbour list of the MD step (pairs within r_c + skin)
    float f_list_cut2;      // (r_c + skin)^2, widened by 1e-5 (the build keeps more, never less)
    float f_half_skin2;     // (skin / 2)^2, narrowed by 1e-5 (a rebuild comes early, never late)
};

// Nose-Hoover state of one system: the friction xi, the velocity update of
// this step, v <- (v a + (dt/m) F) b with a = 1 - xi dt/2, b = 1 / (1 + xi dt/2)
// (FP32: v <- va v + vf F), and the kinetic sum sum m|v|^2 / kT of the step in
// 64-bit fixed point (2^-32), advanced by the prep kernel of the next step.
struct NhState {
    double xi, a, b;
    float f_va, f_vf;
    unsigned long long k2;
    int first;              // 1: the next step keeps xi as it is
    int pad;
};

// A tile of particles of one system: (system, first particle, count, aux).
// aux = first partial index (chunks) or unused (particle blocks).
struct Tile {
    int sys, first, count, aux;
};

// Index checks of the bounds-checked build (compiled with -DRBE_CHECK_BOUNDS):
// RBE_IN_BOUNDS(i, n, err) is true when 0 <= i < n; otherwise it latches
// kErrBounds in the device error word and is false, and the caller skips the
// access.  In the normal build it is the constant true and costs nothing.
#ifdef RBE_CHECK_BOUNDS
__device__ __forceinline__ bool rbe_in_bounds(long long i, long long n, int* err) {
    if (i >= 0 && i < n) return true;
    if (err) atomicOr(err, kErrBounds);
    return false;
}
#define RBE_IN_BOUNDS(i, n, err) ::rbe::rbe_in_bounds((long long)(i), (long long)(n), (err))
#else
#define RBE_IN_BOUNDS(i, n, err) true
#endif

// A warp-aggregated latch of a device condition: the lowest lane that saw it
// sets the bit, one atomic per warp at most.
__device__ __forceinline__ void latch_any(bool cond, int* err, int bit) {
    const unsigned m = __ballot_sync(__activemask(), cond);
    if (m && err && (int)(threadIdx.x & 31) == __ffs(m) - 1) atomicOr(err, bit);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies, the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// ------------------------------------------------- MD update (Sec. 3.3)
// The step's last stage, run by whichever kernel holds a particle's total
// force: the Langevin, Andersen or Nose-Hoover update of its velocity and
// position (caller index o).
//
// Drift r += dt v and wrap into [0, L).
__device__ __forceinline__ void drift_wrap(const SysDev& S, const float4& v, float4& rp) {
    const float L = S.Lf, invL = S.f_invL, dt = S.f_dt;
    rp.x = fmaf(dt, v.x, rp.x); rp.x -= L * floorf(rp.x * invL);
    rp.y = fmaf(dt, v.y, rp.y); rp.y -= L * floorf(rp.y * invL);
    rp.z = fmaf(dt, v.z, rp.z); rp.z -= L * floorf(rp.z * invL);
    // a coordinate just below 0 can round up to exactly L: that is 0
    if (rp.x >= L) rp.x = 0.f;
    if (rp.y >= L) rp.y = 0.f;
    if (rp.z >= L) rp.z = 0.f;
}

// Nose-Hoover leapfrog step on v and rp in registers: v <- va v + vf F (the
// friction taken half before and half after the kick), drift, wrap.  Returns
// m|v|^2/kT in 64-bit fixed point (2^-32) for the kinetic sum of the step.
__device__ __forceinline__ unsigned long long nose_hoover_apply(const SysDev& S, float va,
                                                                float vf, float fx, float fy,
                                                                float fz, float4& v, float4& rp) {
    v.x = fmaf(va, v.x, vf * fx);
    v.y = fmaf(va, v.y, vf * fy);
    v.z = fmaf(va, v.z, vf * fz);
    drift_wrap(S, v, rp);
    const float v2 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
    return __double2ull_rn((double)v2 * S.nh_k2scale);
}

// The same for particle o, from and to memory.
__device__ __forceinline__ unsigned long long nose_hoover_update(float4* md_pos, float4* md_vel,
                                                                 const SysDev& S, float va,
                                                                 float vf, int o, float fx,
                                                                 float fy, float fz) {
    float4 v = md_vel[o];
    float4 rp = md_pos[o];
    const unsigned long long k2 = nose_hoover_apply(S, va, vf, fx, fy, fz, v, rp);
    md_vel[o] = v;
    md_pos[o] = rp;
    return k2;
}

// Sum of a 64-bit value over the warp, added by lane 0 to *dst.
__device__ __forceinline__ void warp_add_u64(unsigned long long v, unsigned long long* dst) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// The thermostat's random numbers for particle o at a step (they do not
// depend on the force, so a kernel may draw them early): Langevin, the normals
// of the Ornstein-Uhlenbeck step; Andersen, the collision test and the new
// velocity's normals.
struct MdNoise {
    float xi0, xi1, xi2;
    bool hit;                                // Andersen collision
};

__device__ __forceinline__ MdNoise md_noise(const SysDev& S, uint64_t step, int o) {
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    const uint32_t pid = (uint32_t)(o - S.off_p);
    const bool andersen = S.thermostat == RBE_THERMO_ANDERSEN;
    // Langevin: normals of the OU step; Andersen: collision word, then normals
    const uint4 c = philox4x32_10(make_uint4(pid, 0u, (uint32_t)step,
                                             (S.stream << 8) | (andersen ? 0x07u : 0x02u)), key);
    MdNoise z{0.f, 0.f, 0.f, andersen && (uint64_t)c.x < S.andersen_thr};
    if (!andersen || z.hit) {
        const uint4 w = andersen ? philox4x32_10(make_uint4(pid, 1u, (uint32_t)step,
                                                            (S.stream << 8) | 0x07u), key)
                                 : c;
        const float u1 = (float)((w.x >> 8) + 1u) * 5.9604644775390625e-08f;   // (0, 1]
        const float u2 = (float)(w.y >> 8) * 5.9604644775390625e-08f;          // [0, 1)
        const float u3 = (float)((w.z >> 8) + 1u) * 5.9604644775390625e-08f;
        const float u4 = (float)(w.w >> 8) * 5.9604644775390625e-08f;
        const float r1 = sqrtf(-2.f * logf(u1)), r3 = sqrtf(-2.f * logf(u3));
        float s2, c2v, s4, c4;
        sincospif(2.f * u2, &s2, &c2v);
        sincospif(2.f * u4, &s4, &c4);
        z.xi0 = r1 * c2v; z.xi1 = r1 * s2; z.xi2 = r3 * c4;
    }
    return z;
}

// Langevin step of Sec. 3.3 (kick, exact Ornstein-Uhlenbeck, drift, wrap) or
// the Andersen loop step (kick, drift, then the collision) on v and rp in
// registers, with total force F and the step's noise z.
__device__ __forceinline__ void md_apply(const SysDev& S, const MdNoise& z, float fx, float fy,
                                         float fz, float4& v, float4& rp) {
    const float dtm = S.f_dt_over_m;
    v.x = fmaf(dtm, fx, v.x);
    v.y = fmaf(dtm, fy, v.y);
    v.z = fmaf(dtm, fz, v.z);
    if (S.thermostat != RBE_THERMO_ANDERSEN) {         // exact Ornstein-Uhlenbeck step
        const float c1 = S.f_c1, c2 = S.f_c2;
        v.x = fmaf(c1, v.x, c2 * z.xi0);
        v.y = fmaf(c1, v.y, c2 * z.xi1);
        v.z = fmaf(c1, v.z, c2 * z.xi2);
    }
    drift_wrap(S, v, rp);
    if (z.hit) {                                        // Andersen collision after the drift
        const float sd = S.f_vsd;
        v.x = sd * z.xi0; v.y = sd * z.xi1; v.z = sd * z.xi2;
    }
}

// Langevin or Andersen step for particle o (caller index) with total force F,
// from and to memory.
__device__ __forceinline__ void langevin_update(float4* md_pos, float4* md_vel,
                                                const uint64_t* cur_step, const SysDev& S, int o,
                                                float fx, float fy, float fz) {
    const MdNoise z = md_noise(S, *cur_step, o);
    float4 v = md_vel[o];
    float4 rp = md_pos[o];
    md_apply(S, z, fx, fy, fz, v, rp);
    md_vel[o] = v;
    md_pos[o] = rp;
}

// Programmatic dependent launch (a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream finishes):
// pdl_wait blocks until every prerequisite grid has completed and its writes
// are visible (it returns at once without one); pdl_trigger lets this grid's
// dependents be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Where a kernel finds its tile of work and its system.  Batch handles pass
// tables (tiles[blockIdx.x], then sysv[tile.sys]); single-system handles pass
// the system's constants by value and the tile size, so a block finds both
// without touching memory (every step starts with cold caches otherwise).
struct Work {
    const SysDev* sysv;   // batch: per-system constants (null for one system)
    const Tile* tiles;    // batch: one tile per block
    int tile;             // one system: particles per block
    int aux_stride;       // one system: tile.aux = blockIdx.x * aux_stride
    SysDev one;           // one system: its constants
};

template <bool ONE>
__device__ __forceinline__ Tile tile_of(const Work& w) {
    if constexpr (ONE) {
        const int first = blockIdx.x * w.tile;
        return Tile{0, first, max(0, min(w.tile, w.one.n - first)),
                    (int)blockIdx.x * w.aux_stride};
    } else {
        return w.tiles[blockIdx.x];
    }
}

// Tile idx of the work (as tile_of, for a block whose index is not the tile's).
template <bool ONE>
__device__ __forceinline__ Tile tile_at(const Work& w, int idx) {
    if constexpr (ONE) {
        const int first = idx * w.tile;
        return Tile{0, first, max(0, min(w.tile, w.one.n - first)), idx * w.aux_stride};
    } else {
        return w.tiles[idx];
    }
}

template <bool ONE>
__device__ __forceinline__ const SysDev& sys_of(const Work& w, int s) {
    if constexpr (ONE) return w.one;
    else return w.sysv[s];
}

// Index of the system owning global item i (start has nsys + 1 entries).
__device__ __forceinline__ int find_sys(const int* __restrict__ start, int nsys, int i) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Smallest j in [0, n) with w < T[j] (T[n-1] = 2^32 > any w).
__device__ __forceinline__ int axis_lookup(const uint64_t* __restrict__ T, int n, uint32_t w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)w < __ldg(T + mid)) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Sample l of system S at `step` (Eq. probexpression, exact inverse CDF per
// axis, (0,0,0) redrawn): (m_x, m_y, m_z, attempts).
__device__ __forceinline__ int4 sample_one(const SysDev& S, const uint64_t* __restrict__ T, int l,
                                           uint64_t step, int* err) {
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    const int n = 2 * S.M + 1;
    for (int a = 0; a < kMaxAttempts; ++a) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)l, (uint32_t)a, (uint32_t)step, (S.stream << 8) | 0x01u), key);
        const int mx = axis_lookup(T, n, w.x) - S.M;
        const int my = axis_lookup(T, n, w.y) - S.M;
        const int mz = axis_lookup(T, n, w.z) - S.M;
        if (mx != 0 || my != 0 || mz != 0) return make_int4(mx, my, mz, a + 1);
    }
    atomicOr(err, kErrSampler);
    return make_int4(1, 0, 0, kMaxAttempts + 1);   // keeps later arithmetic finite
}

// As sample_one, with the tables staged in shared memory as 32-bit words (the
// last entry of each system's table, 2^32, is never read: the search ends at
// index 2M by construction).
__device__ __forceinline__ int4 sample_one_smem(const SysDev& S, const uint32_t* __restrict__ T,
                                                int l, uint64_t step, int* err) {
    const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
    const int last = 2 * S.M;
    auto lookup = [&](uint32_t w) {
        int lo = 0, hi = last;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (w < T[mid]) hi = mid; else lo = mid + 1;
        }
        return lo - S.M;
    };
    for (int a = 0; a < kMaxAttempts; ++a) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)l, (uint32_t)a, (uint32_t)step, (S.stream << 8) | 0x01u), key);
        const int mx = lookup(w.x), my = lookup(w.y), mz = lookup(w.z);
        if (mx != 0 || my != 0 || mz != 0) return make_int4(mx, my, mz, a + 1);
    }
    atomicOr(err, kErrSampler);
    return make_int4(1, 0, 0, kMaxAttempts + 1);
}

// ------------------------------------------------------------- launchers
// `one` selects the single-system kernels (Work.one / Work.tile), else tables.
// cells / sorting (rbe_cells.cu)
// The prep kernels also clear the rho(k) accumulators (2 * nrho words) and,
// with want_q, add each system's charges to qsum_fx (cleared by the caller).
struct PrepArgs {
    double2* blk_q;
    int want_q;
    unsigned long long* qsum_fx;
    unsigned long long* rho_fx;
    int nrho;
    uint64_t* step_dev;
    uint64_t step_arg;
    uint64_t* cur_step;
    // k-batch drawn by the blocks before the particle blocks (one sample per thread)
    int npblk;               // particle blocks; blocks npblk .. draw samples
    int ktot, nsys;
    const int* kstart;       // first sample of each system (nsys + 1)
    const uint64_t* table;
    int tab_words;           // > 0: all tables (this many entries) staged in shared memory
    // the paper's MH sampler: one block per system runs its three chains
    int mh, mh_words;        // mh_words: largest 2M+1 (tables staged per block)
    const uint64_t* mh_tq;
    const double* mh_rho;
    int4* mh_state;
    uint64_t* mh_pos;
    int4* ksamp;
    double* kcoef;           // coef_scale / k^2 per sample (Eq. rbmapprox)
    int* err;
    NhState* nh;             // MD steps: Nose-Hoover state per system (null otherwise)
    // neighbour-list MD steps: displacement test against the last build and
    // the sorted records for the list kernel (null otherwise)
    const uint4* sref;       // [caller index] records at the last build
    const int* iperm;        // caller index -> sorted index of the last build
    uint4* spos;             // [sorted] current records
    int* list_flag;          // set: rebuild the list in this step
    int ncell, ntot;         // cells and particles of all systems (index checks)
};
void launch_prep_mixed(cudaStream_t st, bool one, const Work& w, int nblk, const float4* pos_q,
                       uint4* fx, int* cid, int* rank, int* cell_cnt, const PrepArgs& pa);
void launch_prep_f64(cudaStream_t st, bool one, const Work& w, int nblk, const double4* pos_q,
                     double4* fx64, int* cid, int* rank, int* cell_cnt, const PrepArgs& pa);
// Neighbour-list evaluations: cell ids and slots (cid, rank, cell_cnt) of the
// particles from their fixed-point records, only when *list_flag is set.
void launch_cell_assign(cudaStream_t st, bool one, const Work& w, int nblk, const uint4* fx,
                        int* cid, int* rank, int* cell_cnt, int ncell, const int* list_flag,
                        int* err);
// list_flag (nullable): the cell list is rebuilt only when *list_flag is set
// (the scan returns at once otherwise: no cell was counted).
void launch_scan(cudaStream_t st, int* cell_cnt, int* cell_start, int ncell, uint64_t* step_dev,
                 const uint64_t* cur_step, const int* list_flag = nullptr);
// err (nullable): the device error word, for the index checks of the
// bounds-checked build.
void launch_scatter(cudaStream_t st, int n, const int* cid, const int* rank,
                    const int* cell_start, int* perm_tmp, const int* list_flag = nullptr,
                    int* err = nullptr);
void launch_order(cudaStream_t st, int n, const int* cid, const int* cell_start,
                  const int* perm_tmp, const uint4* fx, uint4* spos, const double4* fx64,
                  double4* spos64, int* perm, const int* list_flag = nullptr,
                  int* iperm = nullptr, int* err = nullptr);

// Neighbour-list build (rbe_real.cu): for every sorted particle the sorted
// indices of the particles within r_c + skin among its 27 neighbour cells.
struct ListArgs {
    Work w;                  // tiles of kBlockP sorted particles
    int nblk;
    const int* list_flag;    // build only when set
    const uint4* spos;
    const int* cell_start;
    int* nbr;                // [slot * stride + i]
    int* ncnt;               // [i]
    int stride, cap;
    uint4* sref;             // the build's records, by caller index (perm)
    const int* perm;         // sorted -> caller index
    unsigned long long* stats;   // [0] builds, [1] largest count
    int* err;
};
void launch_list_build(cudaStream_t st, bool one, const ListArgs& la);

// Fourier part (rbe_fourier.cu).  The structure factors and the Fourier force
// run over the unsorted fixed-point records (caller's order).
void launch_sample(cudaStream_t st, const SysDev* sys, int nsys, int ktot, const int* kstart,
                   const uint64_t* table, const uint64_t* cur_step, int4* ksamp, int* err);
// rho(k) accumulators: 64-bit two's-complement fixed point, scale per system.
__device__ __forceinline__ void rho_accumulate(unsigned long long* dst, double re, double im,
                                               double scale) {
    atomicAdd(dst, (unsigned long long)__double2ll_rn(re * scale));
    atomicAdd(dst + 1, (unsigned long long)__double2ll_rn(im * scale));
}

__device__ __forceinline__ double2 rho_read(const unsigned long long* src, double inv_scale) {
    return make_double2((double)(long long)__ldcg(src) * inv_scale,
                        (double)(long long)__ldcg(src + 1) * inv_scale);
}

// pdl: launched with programmatic stream serialisation (the kernels wait for
// their predecessor's results before reading them).
void launch_rho_mixed(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                      const int4* ksamp, const double* kcoef, const uint4* fx,
                      unsigned long long* rho_fx, int* kcnt, float2* kab, bool pdl = false);
void launch_rho_f64(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                    const int4* ksamp, const double4* fx64, unsigned long long* rho_fx);
// The last stage of a neighbour-list MD step, run by the Fourier-force
// kernel: total force = Fourier + freal, then the thermostat.
struct MdOut {
    const float4* freal;     // real-space force, caller's order (null: no MD stage)
    float4* F_out;           // nullable: total force
    float4* md_pos;          // nullable: positions / velocities updated in place
    float4* md_vel;
    NhState* nh;
    const uint64_t* cur_step;
    int* list_flag;          // nullable: cleared (the step's rebuild flag is consumed)
    // nullable: completion signal of a host-buffer step.  The last block to
    // finish copies the device error word to err_host and then writes the
    // step index after this step (*cur_step + 1) to done_host, both in mapped
    // page-locked memory, after every block's stores are visible system-wide.
    unsigned int* done_cnt;  // blocks finished (device; back to 0 by the last)
    unsigned long long* done_host;
    int* err_host;
    const int* err;
};
void launch_fourier_force_mixed(cudaStream_t st, bool one, const Work& w, int nblk, int split,
                                const uint4* fx, const int4* ksamp, const float2* kab,
                                float4* fs, const MdOut& md = MdOut{}, bool pdl = false);
void launch_fourier_force_f64(cudaStream_t st, bool one, const Work& w, int nblk,
                              const double4* fx64, const int4* ksamp,
                              const unsigned long long* rho_fx, double4* fs64);

// real space, LJ, Langevin, energies (rbe_real.cu)
// Blocks per real-space segment (mixed path): the first takes the particles
// one pass of the block holds, the second the rest (most segments have none,
// and that block returns at once), so a crowded segment does not stretch the
// kernel's tail with a second pass.
constexpr int kSegChunks = 2;

struct RealArgs {
    Work w;                  // real-space tiles of kBlockP / split particles (FP64 path)
    int nrblk;
    int split;               // threads per particle, mixed path (1, 3 or 9)
    int split64;             // threads per particle, FP64 path (power of two)
    int ncell;               // cells over all systems
    int nsys;
    const int* cstart;       // first cell of each system (nsys + 1), batch only
    const Tile* segs;        // mixed path: (system, first cell, cells, packed x0|y<<10|z<<20)
    int nseg;
    int seg_max;             // most cells in one segment
    int stage_cap;           // staged records per segment block
    int seg_threads;         // threads per segment block (64, 128, 192 or 256)
    int parts;               // RBE_PART_* mask
    const int* cell_start;
    const int* perm;
    const uint64_t* cur_step;
    const unsigned long long* qsum_fx;   // per system sum q (fixed point 2^32)
    // mixed
    const uint4* spos;
    const float4* fs;        // Fourier force and dE/dq, caller's order
    float4* F_out;
    float* phi_out;
    float4* md_pos;          // non-null: Langevin update in place
    float4* md_vel;
    // fp64
    const double4* spos64;
    const double4* fs64;
    double4* F_out64;
    double* phi_out64;
    double4* md_pos64;
    double4* md_vel64;
    NhState* nh;             // MD steps: Nose-Hoover state per system
    // neighbour-list MD step (k_real_list): tiles of kBlockP / lsplit sorted
    // particles, lsplit lanes per particle
    Work lw;
    int nlblk, lsplit;
    const int* nbr;
    const int* ncnt;
    int nbr_stride, nbr_cap;
    const int* list_flag;    // rebuild flag of this step
    int list_when;           // the list kernel works only when (*list_flag != 0) == list_when
                             // (2: always)
    int fmode;               // forces call: assemble F, phi, energy and virial partials
    int* flag_clear;         // forces call: the rebuild flag to clear
    float4* freal;           // list kernel output: real-space force, caller's order
    double2* blk_e;          // per block (E_coul, E_lj), nullable
    double2* blk_w;          // per block (W_coul, W_lj): pair virials r.F, nullable
    int* err;                // device error word (index checks of the bounds-checked build)
};
void launch_real_mixed(cudaStream_t st, bool one, const RealArgs& a);
void launch_real_f64(cudaStream_t st, bool one, const RealArgs& a);
void launch_real_list(cudaStream_t st, bool one, const RealArgs& a);
// The MD step's structure factors and its pass over a standing list in one
// launch (rbe_fourier.cu); `a` as for launch_real_list with list_when = 0.
void launch_rho_list(cudaStream_t st, bool one, const Work& w, int nchunks, int ltiles,
                     const int4* ksamp, const double* kcoef, const uint4* fx,
                     unsigned long long* rho_fx, int* kcnt, float2* kab, const RealArgs& a,
                     bool pdl);
void launch_observables(cudaStream_t st, const SysDev& S, const uint4* fx, int first, int n,
                        const int4* mlist, int K, unsigned long long* rho_fx, double2* part,
                        const float4* pos_q, const float4* vel, const double* E_in,
                        const double* W_in, double mass, double* out);
void launch_energy(cudaStream_t st, bool one, const Work& w, int nsys, const int4* ksamp,
                   const unsigned long long* rho_fx, const double2* blk_e,
                   const double2* blk_q, const double2* blk_w, int parts, int per_cell,
                   double* E_out, double* W_out);

}  // namespace rbe
