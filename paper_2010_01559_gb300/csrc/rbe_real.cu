// rbe_real.cu -- real-space Coulomb (Eq. force, second term, truncated at r_c),
// shifted Lennard-Jones (Eq. Ljpotential with r_off = 0), the assembly of the
// total force / dE/dq, the Langevin update of Sec. 3.3, and the FP64 energy
// reduction.
//
// Cells have side >= r_c (+ skin with a neighbour list) and there are at least
// 3 per edge, so every pair within r_c is met exactly once, as the minimum
// image, among the 27 cells around a particle's own.  With r_c > L/3 (up to
// L/2) the box is one cell and every particle meets every other once, again as
// the minimum image.  MD steps on the mixed path walk a Verlet list of the
// pairs within r_c + skin (k_list_build, k_real_list); forces calls scan the
// cells: one block per segment of x-adjacent cells with the neighbourhood
// staged in shared memory and R = 1, 3 or 9 threads per particle, each scanning
// 9/R neighbour rows (k_real_seg).  FP64 path: G threads per particle reading
// the neighbours from global memory.
//
// Real-space pair terms for r < r_c (r_ij = r_j - r_i):
//   F_i   += -lB q_i q_j G(r) r_ij / r,  G = erfc(sqrt(a) r)/r^2 + 2 sqrt(a) e^{-a r^2}/(sqrt(pi) r)
//   phi_i += lB q_j erfc(sqrt(a) r) / r
//   e_i   += lB q_i q_j erfc(sqrt(a) r) / (2 r)
// LJ for r < R_c: F_i -= 24 eps (2 (s/r)^12 - (s/r)^6) r_ij / r^2,
//   e_i += (4 eps ((s/r)^12 - (s/r)^6) + V_shift) / 2.
//
// Langevin (kick, exact Ornstein-Uhlenbeck, drift; m dv = (F - gamma v) dt +
// sqrt(2 gamma kT) dW): v += (dt/m) F; v = c1 v + c2 xi; r = wrap(r + dt v),
// c1 = exp(-gamma dt / m), c2 = sqrt((1 - c1^2) kT / m), xi from Philox with
// counter (i, 0, step_lo, (stream << 8) | 2) by Box-Muller.
// Andersen (the loop of Algorithm 1): v += (dt/m) F; r = wrap(r + dt v); then
// if word 0 of Philox(i, 0, step_lo, (stream << 8) | 7) is below nu dt 2^32,
// v = sqrt(kT/m) xi with xi from Philox(i, 1, step_lo, (stream << 8) | 7).
#include <cmath>

#include "rbe_internal.cuh"
#include "rbe_pair.cuh"
#include "rbe_list_body.cuh"

namespace rbe {



__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// The 27 neighbour cells as 9 rows (dz, dy) of three x-adjacent cells.  Cells
// are numbered x fastest, so a row is one contiguous range of the sorted
// particles unless it wraps around the box edge; then it is two ranges.
__device__ __forceinline__ void row_ranges(const int* __restrict__ cs, int base, int cx, int ncd,
                                           int& s0, int& e0, int& s1, int& e1) {
    if (ncd < 3) {                                  // one cell per edge: the whole row once
        s0 = __ldg(cs + base); e0 = __ldg(cs + base + ncd); s1 = 0; e1 = 0;
    } else if (cx > 0 && cx < ncd - 1) {
        s0 = __ldg(cs + base + cx - 1); e0 = __ldg(cs + base + cx + 2); s1 = 0; e1 = 0;
    } else if (cx == 0) {
        s0 = __ldg(cs + base); e0 = __ldg(cs + base + 2);
        s1 = __ldg(cs + base + ncd - 1); e1 = __ldg(cs + base + ncd);
    } else {
        s0 = __ldg(cs + base + ncd - 2); e0 = __ldg(cs + base + ncd);
        s1 = __ldg(cs + base); e1 = __ldg(cs + base + 1);
    }
}

// ----------------------------------------------------------------- mixed
// One block per cell.  The block stages the records of the 27 neighbouring
// cells (9 rows, each one or two contiguous ranges of the cell-sorted records)
// into shared memory with coalesced loads; then G threads per particle of the
// cell stride over the staged records and combine their sums with shuffles.
// Each thread first runs the cheap distance test over its candidates and keeps
// the indices of those within the cutoff (about one in six) in a list, then
// evaluates erfc / exp / LJ for the listed ones only: a warp whose lanes would
// otherwise take the expensive branch at different candidates now runs it
// densely.  A cell whose neighbourhood exceeds the staging capacity reads the
// records from global memory instead.
constexpr int kNbCap = 24;          // entries of each lane's neighbour list
constexpr int kBatch = 2;           // candidates a thread tests per step of its scan

// Sum of a particle's R lanes (lanes l = 0 .. R-1 of its group), in lane
// order; the result is valid in lane 0 of the group.
template <int R>
__device__ __forceinline__ float lane_combine(float v) {
    float s = v;
#pragma unroll
    for (int d = 1; d < R; ++d) s += __shfl_down_sync(0xffffffffu, v, d);
    return s;
}

// The neighbour rows (r = 3 (dz + 1) + dy + 1) that lane l of a particle's R
// lanes scans, j = 0 .. 9/R - 1.  Along x the centre row reaches r_c on both
// sides, an edge row about 0.79 r_c and a corner row about 0.52 r_c on
// average, so with three lanes the sets {centre, 2 corners}, {2 edges,
// corner}, {2 edges, corner} carry about equal work.
template <int R>
__device__ __forceinline__ int row_of(int l, int j) {
    if constexpr (R == 1) {
        return j;
    } else if constexpr (R == 9) {
        return l;
    } else {
        constexpr unsigned long long tab = 4ull | (0ull << 4) | (8ull << 8) | (1ull << 12) |
                                           (7ull << 16) | (2ull << 20) | (3ull << 24) |
                                           (5ull << 28) | (6ull << 32);
        return (int)((tab >> (4 * (3 * l + j))) & 15ull);
    }
}

// Corner of cell c along an axis, floor(c 2^32 / ncd), from the system's
// quotient and remainder of 2^32 / ncd (c = ncd wraps to 0).  Every fixed-point
// coordinate of cell c lies in [corner(c), corner(c + 1)), so integer
// differences to corners bound the distance to any record of a neighbour cell
// from below, exactly.
__device__ __forceinline__ uint32_t corner_of(int c, const SysDev& S) {
    return (uint32_t)c * S.corner_q + ((uint32_t)c * S.corner_r) / (uint32_t)S.ncd;
}


// One block per segment: nsc x-adjacent cells of one (y, z) row.  The block
// copies, for each of the 9 neighbour rows, the segment's cells plus one halo
// cell on each side into shared memory (fixed-point records, each cell's
// records in ascending x); per-cell boundaries of the staged rows go to a small
// table.  A particle in cell x finds its 27 neighbour cells as 9 contiguous
// windows of three cells, ascending in x.  The y and z distances from the
// particle to a row's cells bound what is left of the cutoff along x, so the
// window shrinks to the records within that reach: whole rows and halo cells
// drop out, and the scan stops at the first record past the reach (cells of
// at least 5 per edge keep the 3-cell window below half the box, where the
// 32-bit differences are monotone).  Each of a particle's R threads (adjacent
// lanes of one warp) scans its own rows, lists the records within the cutoff
// and then evaluates erfc / exp / LJ densely for the listed ones; the R
// partial sums are added in lane order.  A segment whose neighbourhood exceeds
// the staging buffer reads its candidates from global memory instead.
template <int R, bool ONE, int NT>
__global__ void __launch_bounds__(NT, (NT == 192 ? 5 : 1024 / NT))
k_real_seg(const __grid_constant__ RealArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* s_rec = (uint4*)smem;                                      // [stage_cap]
    uint16_t* s_nb = (uint16_t*)(s_rec + a.stage_cap);                // [kNbCap][NT]
    int* s_b = (int*)(s_nb + kNbCap * NT);                            // [9][seg_max + 3]
    uint32_t* s_cx = (uint32_t*)(s_b + 9 * (a.seg_max + 3));          // [seg_max + 1]
    __shared__ int s_src[27], s_len[27], s_off[28];
    constexpr int PPW = 32 / R;                  // particles per warp (R = 3: two lanes idle)
    constexpr int NW = NT / 32;
    constexpr int RPL = 9 / R;                   // neighbour rows per lane
    const int chunk = blockIdx.x % kSegChunks;
    const Tile sg = a.segs[blockIdx.x / kSegChunks];
    const int sys = sg.sys;
    const SysDev& S = sys_of<ONE>(a.w, sys);
    const int ncd = S.ncd;
    const int nsc = sg.count;                                         // cells in the segment
    const int x0 = sg.aux & 1023, cy = (sg.aux >> 10) & 1023, cz = (sg.aux >> 20) & 1023;
    const int x1 = x0 + nsc - 1;
    const int bstride = a.seg_max + 3;
    const int seg_s = __ldg(a.cell_start + sg.first), seg_e = __ldg(a.cell_start + sg.first + nsc);
    // this block's share of the segment's particles: one pass, or the rest
    const int own_s = seg_s + (chunk == 0 ? 0 : NW * PPW);
    const int own_e = chunk == 0 ? min(seg_e, seg_s + NW * PPW) : seg_e;
    const int nown = max(0, own_e - own_s);
    if (chunk > 0 && nown == 0) {                 // nothing beyond the first pass
        if (a.blk_e && threadIdx.x == 0) a.blk_e[blockIdx.x] = make_double2(0.0, 0.0);
        if (a.blk_w && threadIdx.x == 0) a.blk_w[blockIdx.x] = make_double2(0.0, 0.0);
        return;
    }
    const bool do_real = (a.parts & kPartReal) != 0;
    const bool do_lj = (a.parts & kPartLJ) != 0 && S.lj_eps != 0.0;
    const bool pairs = nown > 0 && (do_real || do_lj);
    const bool nhm = a.md_pos && a.nh && S.thermostat == RBE_THERMO_NOSE_HOOVER;
    float nh_va = 0.f, nh_vf = 0.f;
    if (nhm) {
        nh_va = a.nh[sys].f_va;
        nh_vf = a.nh[sys].f_vf;
    }
    const float Lu = S.L_over_2_32;
    for (int j = threadIdx.x; j <= nsc; j += blockDim.x) s_cx[j] = corner_of(x0 + j, S);
    if (pairs && threadIdx.x < 27) {
        const int r = threadIdx.x / 3, part = threadIdx.x % 3;
        const int zz = wrapc(cz + r / 3 - 1, ncd), yy = wrapc(cy + r % 3 - 1, ncd);
        const int row = S.off_c + (zz * ncd + yy) * ncd;
        int b, e;
        if (part == 1) {
            b = __ldg(a.cell_start + row + x0);
            e = __ldg(a.cell_start + row + x1 + 1);
        } else {
            const int xh = wrapc(part == 0 ? x0 - 1 : x1 + 1, ncd);
            b = __ldg(a.cell_start + row + xh);
            e = __ldg(a.cell_start + row + xh + 1);
        }
        s_src[threadIdx.x] = b;
        s_len[threadIdx.x] = e - b;
    }
    __syncthreads();
    if (pairs && threadIdx.x < 32) {
        const int v = threadIdx.x < 27 ? s_len[threadIdx.x] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)threadIdx.x >= o) incl += y;
        }
        if (threadIdx.x < 27) s_off[threadIdx.x + 1] = incl;
        if (threadIdx.x == 0) s_off[0] = 0;
    }
    __syncthreads();
    const int total = pairs ? s_off[27] : 0;
    const bool staged = total <= a.stage_cap;
    if (pairs) {
        // window boundaries: row r, boundary j of cells x0-1 .. x1+1 (j = 0 .. nsc+2)
        for (int idx = threadIdx.x; idx < 9 * (nsc + 3); idx += blockDim.x) {
            const int r = idx / (nsc + 3), j = idx - r * (nsc + 3);
            int v;
            if (j == 0) {
                v = s_off[3 * r];
            } else if (j <= nsc + 1) {
                const int zz = wrapc(cz + r / 3 - 1, ncd), yy = wrapc(cy + r % 3 - 1, ncd);
                const int row = S.off_c + (zz * ncd + yy) * ncd;
                v = s_off[3 * r + 1] + (__ldg(a.cell_start + row + x0 + j - 1) - s_src[3 * r + 1]);
            } else {
                v = s_off[3 * r + 3];
            }
            s_b[r * bstride + j] = v;
        }
        if (staged)
            // every thread issues its loads at once: staged slot k comes from
            // range q (binary search over the prefix), consecutive k consecutive
            for (int k = threadIdx.x; k < total; k += blockDim.x) {
                int lo = 0, hi = 26;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= k) lo = mid; else hi = mid - 1;
                }
                s_rec[k] = __ldg(a.spos + s_src[lo] + (k - s_off[lo]));
            }
    }
    __syncthreads();
    PairConst kc;
    kc.rc2 = do_real ? S.f_rc2 : 0.f;
    kc.lj_rc2 = do_lj ? S.f_lj_rc2 : 0.f;
    kc.alpha = S.f_alpha;
    kc.sa = S.f_sqrt_alpha;
    kc.two_sa_spi = S.f_two_sa_spi;
    kc.lB = S.f_lB;
    kc.lj_s2 = S.f_lj_sigma2;
    kc.lj_eps = S.f_lj_eps;
    kc.lj_shift = S.f_lj_shift;
    kc.vir = a.blk_w != nullptr;
    const float cut2 = fmaxf(kc.rc2, kc.lj_rc2);
    const float invLu = S.f_inv_Lu;
    // distance test in fixed-point units; the margins keep the test and the
    // reach conservative against FP32 rounding (pair_terms applies the cutoffs)
    const float cut2u = cut2 * invLu * invLu * 1.00001f;
    const float reach_slack = cut2 * 1e-5f;
    const bool prune = ncd >= 5;
    const uint32_t ylo = corner_of(cy, S), yhi = corner_of(cy + 1, S);
    const uint32_t zlo = corner_of(cz, S), zhi = corner_of(cz + 1, S);
    const bool want_phi = a.phi_out != nullptr;
    const bool want_e = a.blk_e != nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pl = lane / R, l = lane - pl * R;  // particle of the warp, lane within it
    double ec_own = 0.0, elj_own = 0.0, wc_own = 0.0, wlj_own = 0.0;
    constexpr int kPass = NW * PPW;              // particles per pass of the block
    __shared__ float4 s_f[kPass];                // a pass's real-space force and phi
    for (int pass = 0; pass < nown; pass += kPass) {
        const int base = pass + warp * PPW;
        const bool active = pl < PPW && base + pl < nown;
        const int i = own_s + min(base + pl, nown - 1);
        const uint4 si = a.spos[i];
        const int cxi = (int)(((unsigned long long)si.x * (unsigned long long)ncd) >> 32);
        const float lbqi = kc.lB * __uint_as_float(si.w);
        PairAcc acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (active && pairs) {
            const int u = cxi - x0;                       // 0 .. nsc-1
            if (staged) {
                // distances to the faces of the particle's cell: squared in
                // length units for y and z, fixed-point for x
                const float fyl = (float)(si.y - ylo) * Lu, fyh = (float)(yhi - si.y) * Lu;
                const float fzl = (float)(si.z - zlo) * Lu, fzh = (float)(zhi - si.z) * Lu;
                const float fyl2 = fyl * fyl, fyh2 = fyh * fyh, fzl2 = fzl * fzl, fzh2 = fzh * fzh;
                const uint32_t oxl = si.x - s_cx[u], oxh = s_cx[u + 1] - si.x;
                int cnt = 0;
#pragma unroll 1
                for (int jr = 0; jr < RPL; ++jr) {
                    const int r = row_of<R>(l, jr);
                    const int ry = r % 3, rz = r / 3;
                    const float reach2 = cut2 + reach_slack -
                                         (ry == 0 ? fyl2 : (ry == 2 ? fyh2 : 0.f)) -
                                         (rz == 0 ? fzl2 : (rz == 2 ? fzh2 : 0.f));
                    if (reach2 <= 0.f) continue;          // the whole row is beyond the cutoff
                    if (ncd == 1 && r != 4) continue;     // one cell per edge: own cell once
                    const int* bb = s_b + r * bstride + u;
                    int kb = ncd == 1 ? bb[1] : bb[0], ke = ncd == 1 ? bb[2] : bb[3];
                    int w = 0x7FFFFFFF;                   // no x limit below 5 cells per edge
                    if (prune) {
                        w = (int)(sqrtf(reach2) * invLu) + 8;
                        if (oxl > (uint32_t)w) kb = bb[1];    // cell x-1 out of reach
                        if (oxh > (uint32_t)w) ke = bb[2];    // cell x+1 out of reach
                    }
                    const uint32_t wu = (uint32_t)w;
                    // batches of kBatch consecutive records: the shared-memory
                    // loads of a batch are independent and overlap
                    for (int k0 = kb; k0 < ke; k0 += kBatch) {
                        uint4 sj[kBatch];
#pragma unroll
                        for (int q = 0; q < kBatch; ++q) sj[q] = s_rec[min(k0 + q, ke - 1)];
                        bool past = false;
#pragma unroll
                        for (int q = 0; q < kBatch; ++q) {
                            const int k = k0 + q;
                            const int dxi = (int)(sj[q].x - si.x);
                            past |= dxi > w;
                            if (k < ke && (uint32_t)dxi + wu <= 2u * wu) {   // |dxi| <= w
                                const float dx = (float)dxi;
                                const float dy = (float)(int32_t)(sj[q].y - si.y);
                                const float dz = (float)(int32_t)(sj[q].z - si.z);
                                const float r2u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                if (r2u < cut2u && r2u > 0.f) {
                                    if (cnt < kNbCap) s_nb[cnt++ * NT + threadIdx.x] = (uint16_t)k;
                                    else pair_fixed(si, sj[q], Lu, lbqi, kc, acc);
                                }
                            }
                        }
                        if (past) break;                   // ascending x: the rest is beyond
                    }
                }
                for (int e = 0; e < cnt; ++e) {
                    const uint4 sj = s_rec[s_nb[e * NT + threadIdx.x]];
                    pair_fixed(si, sj, Lu, lbqi, kc, acc);
                }
            } else {
                // candidates straight from the cell-sorted records
                for (int jr = 0; jr < RPL; ++jr) {
                    const int r = row_of<R>(l, jr);
                    if (ncd == 1 && r != 4) continue;     // one cell per edge: own cell once
                    const int zz = wrapc(cz + r / 3 - 1, ncd), yy = wrapc(cy + r % 3 - 1, ncd);
                    const int row = S.off_c + (zz * ncd + yy) * ncd;
                    for (int d = (ncd == 1 ? 0 : -1); d <= (ncd == 1 ? 0 : 1); ++d) {
                        const int xn = wrapc(cxi + d, ncd);
                        const int cb = __ldg(a.cell_start + row + xn);
                        const int ce = __ldg(a.cell_start + row + xn + 1);
                        for (int j = cb; j < ce; ++j) {
                            if (j == i) continue;
                            pair_fixed(si, __ldg(a.spos + j), Lu, lbqi, kc, acc);
                        }
                    }
                }
            }
        }
        acc.fx = lane_combine<R>(acc.fx);
        acc.fy = lane_combine<R>(acc.fy);
        acc.fz = lane_combine<R>(acc.fz);
        if (want_phi) acc.phr = lane_combine<R>(acc.phr);
        if (want_e) {
            acc.ec = lane_combine<R>(acc.ec);
            acc.elj = lane_combine<R>(acc.elj);
        }
        if (kc.vir) {
            acc.wc = lane_combine<R>(acc.wc);
            acc.wlj = lane_combine<R>(acc.wlj);
        }
        if (active && l == 0) {
            s_f[warp * PPW + pl] = make_float4(acc.fx, acc.fy, acc.fz, acc.phr);
            if (want_e) {
                ec_own += (double)acc.ec;
                elj_own += (double)acc.elj;
            }
            if (kc.vir) {
                wc_own += (double)acc.wc;
                wlj_own += (double)acc.wlj;
            }
        }
        __syncthreads();
        // the rest runs one thread per particle: total force, outputs, Langevin
        const int np = min(kPass, nown - pass);
        unsigned long long k2 = 0ull;
        if ((int)threadIdx.x < np) {
            const int i = own_s + pass + threadIdx.x;
            const int o = a.perm[i];
            const float4 fr = s_f[threadIdx.x];
            float fx = fr.x, fy = fr.y, fz = fr.z, phi = fr.w;
            if (a.parts & kPartFourier) {
                const float4 f = a.fs[o];
                fx += f.x; fy += f.y; fz += f.z;
                if (want_phi) {
                    const double qi = (double)__uint_as_float(a.spos[i].w);
                    const double qs = (double)(long long)__ldcg(a.qsum_fx + sys) / kQScale;
                    phi += f.w - (float)(2.0 * S.self_coef * qi + S.bg_coef * qs);
                }
            }
            if (a.F_out) a.F_out[o] = make_float4(fx, fy, fz, 0.f);
            if (want_phi) a.phi_out[o] = phi;
            if (nhm) k2 = nose_hoover_update(a.md_pos, a.md_vel, S, nh_va, nh_vf, o, fx, fy, fz);
            else if (a.md_pos) langevin_update(a.md_pos, a.md_vel, a.cur_step, S, o, fx, fy, fz);
        }
        if (nhm) warp_add_u64(k2, &a.nh[sys].k2);
        __syncthreads();
    }
    if (want_e) {
        const double2 r = block_sum2_real(ec_own, elj_own);
        if (threadIdx.x == 0) a.blk_e[blockIdx.x] = r;
    }
    if (kc.vir) {
        __syncthreads();                                // the partial buffers are reused
        const double2 r = block_sum2_real(wc_own, wlj_own);
        if (threadIdx.x == 0) a.blk_w[blockIdx.x] = r;
    }
}

// ----------------------------------------------------------- neighbour list
// Verlet list of the MD step: the pairs within r_c + skin, rebuilt only when
// some particle has moved more than skin/2 since the last build (the prep
// kernel tests that), so every pair within r_c stays in the list between
// builds.  Cells have side >= r_c + skin.

// One thread per sorted particle: the 27 neighbour cells as 9 rows of three
// x-adjacent cells (one row, once, with one cell per edge), every j != i whose
// fixed-point minimum-image distance is within r_c + skin, in scan order.  The
// record of the build is kept, by caller index, as the reference of the
// displacement test.
template <bool ONE>
__global__ void __launch_bounds__(kBlockP) k_list_build(const __grid_constant__ ListArgs la) {
    if (!*la.list_flag) return;
    const Tile tl = tile_of<ONE>(la.w);
    const SysDev& S = sys_of<ONE>(la.w, tl.sys);
    const int t = threadIdx.x;
    int cnt = 0;
    if (t < tl.count) {
        const int i = tl.first + t;
        const uint4 si = la.spos[i];
        const int ncd = S.ncd;
        const int cx = (int)(((unsigned long long)si.x * (unsigned long long)ncd) >> 32);
        const int cy = (int)(((unsigned long long)si.y * (unsigned long long)ncd) >> 32);
        const int cz = (int)(((unsigned long long)si.z * (unsigned long long)ncd) >> 32);
        const float Lu = S.L_over_2_32, cut2 = S.f_list_cut2;
        const int dlo = ncd < 3 ? 0 : -1, dhi = ncd < 3 ? 0 : 1;
        int* out = la.nbr + i;
        const size_t stride = (size_t)la.stride;
        // one sweep: the pairs within r_c go to the front of the particle's
        // slots, those in the skin to the back; the skin block then moves up
        // behind the first, so that the lanes of a warp in the list pass mostly
        // agree on the cutoff branch at the same position in their lists
        const float rc2 = S.f_rc2;
        int n_in = 0, n_sk = 0;
        for (int dz = dlo; dz <= dhi; ++dz) {
            for (int dy = dlo; dy <= dhi; ++dy) {
                const int zz = wrapc(cz + dz, ncd), yy = wrapc(cy + dy, ncd);
                int r0, e0, r1, e1;
                row_ranges(la.cell_start, S.off_c + (zz * ncd + yy) * ncd, cx, ncd, r0, e0, r1, e1);
                for (int part = 0; part < 2; ++part) {
                    const int b = part ? r1 : r0, e = part ? e1 : e0;
                    for (int j = b; j < e; ++j) {
                        if (!RBE_IN_BOUNDS(j, la.stride, la.err)) break;
                        const uint4 sj = __ldg(la.spos + j);
                        const float dx = (float)(int32_t)(sj.x - si.x) * Lu;
                        const float dyy = (float)(int32_t)(sj.y - si.y) * Lu;
                        const float dzz = (float)(int32_t)(sj.z - si.z) * Lu;
                        const float r2 = fmaf(dx, dx, fmaf(dyy, dyy, dzz * dzz));
                        if (r2 < cut2 && j != i) {
                            if (n_in + n_sk < la.cap) {
                                const int slot = r2 < rc2 ? n_in : la.cap - 1 - n_sk;
                                out[(size_t)slot * stride] = j;
                            }
                            if (r2 < rc2) ++n_in; else ++n_sk;
                        }
                    }
                }
            }
        }
        cnt = n_in + n_sk;
        if (cnt <= la.cap) {
            // move the skin block [cap - n_sk, cap) to [n_in, n_in + n_sk);
            // the destination never lies above the source: ascending is safe
            for (int k = 0; k < n_sk; ++k)
                out[(size_t)(n_in + k) * stride] = out[(size_t)(la.cap - n_sk + k) * stride];
        }
        la.ncnt[i] = min(cnt, la.cap);
        const int o = la.perm[i];
        if (RBE_IN_BOUNDS(o, la.stride, la.err))
            la.sref[o] = si;                // by caller index: the prep kernel reads it in order
        if (cnt > la.cap) atomicOr(la.err, kErrList);
    }
    const unsigned wmax = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
    if ((t & 31) == 0 && wmax) atomicMax(la.stats + 1, (unsigned long long)wmax);
    if (blockIdx.x == 0 && t == 0) atomicAdd(la.stats, 1ull);
}

// ----------------------------------------------------------------- FP64
template <int G, bool ONE>
__global__ void __launch_bounds__(kBlockP)
k_real_f64(const __grid_constant__ RealArgs a) {
    const Tile tl = tile_of<ONE>(a.w);
    const SysDev& S = sys_of<ONE>(a.w, tl.sys);
    const int g = threadIdx.x % G;
    const int t = threadIdx.x / G;
    const bool active = t < tl.count;
    const int i = tl.first + (tl.count > 0 ? min(t, tl.count - 1) : 0);
    double4 pi = make_double4(0, 0, 0, 0);
    if (tl.count > 0) pi = a.spos64[i];
    const double qi = pi.w;
    const bool do_real = (a.parts & kPartReal) != 0;
    const bool do_lj = (a.parts & kPartLJ) != 0 && S.lj_eps != 0.0;
    double fx = 0, fy = 0, fz = 0, phr = 0, ec = 0, elj = 0, wc = 0, wlj = 0;
    const bool vir = a.blk_w != nullptr;
    if (active && (do_real || do_lj)) {
        const int ncd = S.ncd;
        auto cell = [&](double w) {
            const double u = w * S.invL * (double)ncd;
            return (u >= 0.0 && u < (double)ncd) ? (int)u : 0;
        };
        const int cx = cell(pi.x), cy = cell(pi.y), cz = cell(pi.z);
        const double L = S.L, invL = S.invL;
        const double rc2 = do_real ? S.r_c * S.r_c : 0.0;
        const double lj_rc2 = do_lj ? S.lj_rcut2 : 0.0;
        const double two_sa_spi = 2.0 * S.sqrt_alpha / sqrt(M_PI);
        const int dlo = ncd < 3 ? 0 : -1, dhi = ncd < 3 ? 0 : 1;   // one cell: all pairs once
        for (int dz = dlo; dz <= dhi; ++dz) {
            const int zz = wrapc(cz + dz, ncd);
            for (int dy = dlo; dy <= dhi; ++dy) {
                const int yy = wrapc(cy + dy, ncd);
                int s0, e0, s1, e1;
                row_ranges(a.cell_start, S.off_c + (zz * ncd + yy) * ncd, cx, ncd, s0, e0, s1, e1);
                for (int r = 0; r < 2; ++r) {
                    const int s = r ? s1 : s0, e = r ? e1 : e0;
                    for (int j = s + g; j < e; j += G) {
                        if (j == i) continue;
                        const double4 pj = a.spos64[j];
                        double ddx = pj.x - pi.x, ddy = pj.y - pi.y, ddz = pj.z - pi.z;
                        ddx -= L * rint(ddx * invL);
                        ddy -= L * rint(ddy * invL);
                        ddz -= L * rint(ddz * invL);
                        const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        if (r2 < rc2) {
                            const double r = sqrt(r2);
                            const double erfc_v = erfc(S.sqrt_alpha * r);
                            const double G_ = erfc_v / r2 + two_sa_spi * exp(-S.alpha * r2) / r;
                            const double s_ = -S.lB * qi * pj.w * G_ / r;
                            fx += s_ * ddx; fy += s_ * ddy; fz += s_ * ddz;
                            phr += S.lB * pj.w * erfc_v / r;
                            ec += 0.5 * S.lB * qi * pj.w * erfc_v / r;
                            if (vir)
                                wc += 0.5 * S.lB * qi * pj.w *
                                      (erfc_v / r + two_sa_spi * exp(-S.alpha * r2));
                        }
                        if (r2 < lj_rc2) {
                            const double sr2 = S.lj_sigma2 / r2;
                            const double sr6 = sr2 * sr2 * sr2;
                            const double mag = 24.0 * S.lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                            fx -= mag * ddx; fy -= mag * ddy; fz -= mag * ddz;
                            elj += 0.5 * (4.0 * S.lj_eps * (sr6 * sr6 - sr6) + S.lj_shift);
                            if (vir) wlj += 0.5 * mag * r2;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o, G);
        fy += __shfl_down_sync(0xffffffffu, fy, o, G);
        fz += __shfl_down_sync(0xffffffffu, fz, o, G);
        phr += __shfl_down_sync(0xffffffffu, phr, o, G);
        ec += __shfl_down_sync(0xffffffffu, ec, o, G);
        elj += __shfl_down_sync(0xffffffffu, elj, o, G);
        wc += __shfl_down_sync(0xffffffffu, wc, o, G);
        wlj += __shfl_down_sync(0xffffffffu, wlj, o, G);
    }
    const bool owner = active && g == 0;
    if (owner) {
        double phi = phr;
        const int o = a.perm[i];
        if (a.parts & kPartFourier) {
            const double4 f = a.fs64[o];
            fx += f.x; fy += f.y; fz += f.z;
            if (a.phi_out64) {
                const double qs = (double)(long long)__ldcg(a.qsum_fx + tl.sys) / kQScale;
                phi += f.w - 2.0 * S.self_coef * qi - S.bg_coef * qs;
            }
        }
        if (a.F_out64) a.F_out64[o] = make_double4(fx, fy, fz, 0.0);
        if (a.phi_out64) a.phi_out64[o] = phi;
        if (a.md_pos64 && a.nh && S.thermostat == RBE_THERMO_NOSE_HOOVER) {
            // Nose-Hoover leapfrog: v <- (v a + (dt/m) F) b, drift, wrap
            const double na = a.nh[tl.sys].a, nb = a.nh[tl.sys].b;
            const double F3[3] = {fx, fy, fz};
            double4 v = a.md_vel64[o];
            double4 rp = a.md_pos64[o];
            double* vv[3] = {&v.x, &v.y, &v.z};
            double* rr[3] = {&rp.x, &rp.y, &rp.z};
            double v2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double vd = (*vv[d] * na + S.dt_over_m * F3[d]) * nb;
                double rd = *rr[d] + S.dt * vd;
                rd -= S.L * floor(rd / S.L);
                *vv[d] = vd;
                *rr[d] = rd;
                v2 += vd * vd;
            }
            a.md_vel64[o] = v;
            a.md_pos64[o] = rp;
            atomicAdd(&a.nh[tl.sys].k2, __double2ull_rn(v2 * S.nh_k2scale));
        } else if (a.md_pos64) {
            const uint64_t step = *a.cur_step;
            const uint2 key = make_uint2((uint32_t)S.seed, (uint32_t)(S.seed >> 32));
            const uint32_t pid = (uint32_t)(o - S.off_p);
            const bool andersen = S.thermostat == RBE_THERMO_ANDERSEN;
            // Langevin: normals of the OU step; Andersen: collision word, then normals
            const uint4 c = philox4x32_10(make_uint4(pid, 0u, (uint32_t)step,
                                                     (S.stream << 8) | (andersen ? 0x07u : 0x02u)),
                                          key);
            const bool hit = andersen && (uint64_t)c.x < S.andersen_thr;
            const uint4 w = andersen ? philox4x32_10(make_uint4(pid, 1u, (uint32_t)step,
                                                                (S.stream << 8) | 0x07u), key)
                                     : c;
            const double u1 = ((double)w.x + 1.0) / 4294967296.0;
            const double u2 = (double)w.y / 4294967296.0;
            const double u3 = ((double)w.z + 1.0) / 4294967296.0;
            const double u4 = (double)w.w / 4294967296.0;
            const double r1 = sqrt(-2.0 * log(u1)), r3 = sqrt(-2.0 * log(u3));
            const double xi[3] = {r1 * cos(2.0 * M_PI * u2), r1 * sin(2.0 * M_PI * u2),
                                  r3 * cos(2.0 * M_PI * u4)};
            const double F3[3] = {fx, fy, fz};
            double4 v = a.md_vel64[o];
            double4 rp = a.md_pos64[o];
            double* vv[3] = {&v.x, &v.y, &v.z};
            double* rr[3] = {&rp.x, &rp.y, &rp.z};
            const double L = S.L;
            for (int d = 0; d < 3; ++d) {
                double vd = *vv[d] + S.dt_over_m * F3[d];
                if (!andersen) vd = S.c1 * vd + S.c2 * xi[d];
                double rd = *rr[d] + S.dt * vd;
                rd -= L * floor(rd / L);
                if (hit) vd = S.vsd * xi[d];           // Andersen collision after the drift
                *vv[d] = vd;
                *rr[d] = rd;
            }
            a.md_vel64[o] = v;
            a.md_pos64[o] = rp;
        }
    }
    if (a.blk_e) {
        const double2 r = block_sum2_real(owner ? ec : 0.0, owner ? elj : 0.0);
        if (threadIdx.x == 0) a.blk_e[blockIdx.x] = r;
    }
    if (vir) {
        __syncthreads();                                // the partial buffers are reused
        const double2 r = block_sum2_real(owner ? wc : 0.0, owner ? wlj : 0.0);
        if (threadIdx.x == 0) a.blk_w[blockIdx.x] = r;
    }
}

// ----------------------------------------------------------------- energy
// One block per system: fixed-order FP64 sums of the per-k energy terms and the
// per-block real-space / LJ partials, plus the self and background terms.
// One block per system, fixed-order FP64 sums: the estimator's Fourier terms
// (S/P) 2 pi |rho(k)|^2 / (V k^2) from the fixed-point accumulators, the
// self and background terms from the per-block charge sums, and the
// real-space partials (per cell on the mixed path, per block on the FP64 one).
template <bool ONE>
__global__ void k_energy(const __grid_constant__ Work w, const int4* __restrict__ ksamp,
                         const unsigned long long* __restrict__ rho_fx,
                         const double2* __restrict__ blk_e, const double2* __restrict__ blk_q,
                         const double2* __restrict__ blk_w, int parts, int per_cell,
                         double* __restrict__ E_out, double* __restrict__ W_out) {
    const SysDev& S = sys_of<ONE>(w, blockIdx.x);
    double ef = 0.0, ec = 0.0, elj = 0.0, q1 = 0.0, q2 = 0.0;
    if (parts & kPartFourier) {
        const double tp = 2.0 * M_PI * S.invL;
        for (int l = threadIdx.x; l < S.P; l += blockDim.x) {
            const int4 m = ksamp[S.off_k + l];
            const double2 r = rho_read(rho_fx + 2 * (S.off_k + l), S.rho_inv_scale);
            const double k2 = tp * tp * ((double)m.x * m.x + (double)m.y * m.y + (double)m.z * m.z);
            ef += 0.5 * (S.coef_scale / k2) * (r.x * r.x + r.y * r.y);
        }
        for (int b = threadIdx.x; b < S.nb; b += blockDim.x) {
            const double2 v = blk_q[S.off_b + b];
            q1 += v.x;
            q2 += v.y;
        }
    }
    // partials per FP64 block (0), per segment block (1) or per list block (2)
    const int off = per_cell == 2 ? S.off_lb : (per_cell ? S.off_sg * kSegChunks : S.off_rb);
    const int nb = per_cell == 2 ? S.nlb : (per_cell ? S.nsg * kSegChunks : S.nrb);
    double wc = 0.0, wlj = 0.0;
    if (blk_e)
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const double2 v = blk_e[off + b];
            ec += v.x;
            elj += v.y;
        }
    if (blk_w)
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const double2 v = blk_w[off + b];
            wc += v.x;
            wlj += v.y;
        }
    __shared__ double sf[256], sc[256], sl[256], s1[256], s2[256], sw[256], sv[256];
    sf[threadIdx.x] = ef; sc[threadIdx.x] = ec; sl[threadIdx.x] = elj;
    s1[threadIdx.x] = q1; s2[threadIdx.x] = q2;
    sw[threadIdx.x] = wc; sv[threadIdx.x] = wlj;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sf[threadIdx.x] += sf[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
            sl[threadIdx.x] += sl[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
            sw[threadIdx.x] += sw[threadIdx.x + o];
            sv[threadIdx.x] += sv[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double Ef = 0.0;
        if (parts & kPartFourier)
            Ef = sf[0] - S.self_coef * s2[0] - 0.5 * S.bg_coef * s1[0] * s1[0];
        const double Ec = (parts & kPartReal) ? sc[0] : 0.0;
        const double El = (parts & kPartLJ) ? sl[0] : 0.0;
        E_out[4 * blockIdx.x + 0] = Ef + Ec + El;
        E_out[4 * blockIdx.x + 1] = Ef;
        E_out[4 * blockIdx.x + 2] = Ec;
        E_out[4 * blockIdx.x + 3] = El;
        if (W_out) {                                    // real-space Coulomb and LJ virials
            W_out[2 * blockIdx.x + 0] = (parts & kPartReal) ? sw[0] : 0.0;
            W_out[2 * blockIdx.x + 1] = (parts & kPartLJ) ? sv[0] : 0.0;
        }
    }
}

// Dynamic shared memory of the segment kernel for a staging capacity.
size_t real_seg_smem(int stage_cap, int seg_max, int nt) {
    return sizeof(uint4) * (size_t)stage_cap + sizeof(uint16_t) * kNbCap * (size_t)nt +
           sizeof(int) * 9 * (size_t)(seg_max + 3) + sizeof(uint32_t) * (size_t)(seg_max + 1);
}

template <int R, int NT>
static void real_mixed_rn(cudaStream_t st, bool one, const RealArgs& a) {
    const size_t smem = real_seg_smem(a.stage_cap, a.seg_max, NT);
    if (one) {
        cudaFuncSetAttribute(k_real_seg<R, true, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_real_seg<R, true, NT><<<a.nseg * kSegChunks, NT, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_real_seg<R, false, NT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_real_seg<R, false, NT><<<a.nseg * kSegChunks, NT, smem, st>>>(a);
    }
}

// Block size: enough warps for the particles of a typical segment, 64 .. 256.
template <int R>
static void real_mixed_r(cudaStream_t st, bool one, const RealArgs& a) {
    if (a.seg_threads >= 256) real_mixed_rn<R, 256>(st, one, a);
    else if (a.seg_threads >= 192) real_mixed_rn<R, 192>(st, one, a);
    else if (a.seg_threads >= 128) real_mixed_rn<R, 128>(st, one, a);
    else real_mixed_rn<R, 64>(st, one, a);
}

template <int G>
static void real_f64_g(cudaStream_t st, bool one, const RealArgs& a) {
    if (one) k_real_f64<G, true><<<a.nrblk, kBlockP, 0, st>>>(a);
    else k_real_f64<G, false><<<a.nrblk, kBlockP, 0, st>>>(a);
}

void launch_real_mixed(cudaStream_t st, bool one, const RealArgs& a) {
    if (a.nseg <= 0) return;
    switch (a.split) {
        case 3: real_mixed_r<3>(st, one, a); break;
        case 9: real_mixed_r<9>(st, one, a); break;
        default: real_mixed_r<1>(st, one, a); break;
    }
}

template <int R>
static void real_list_r(cudaStream_t st, bool one, const RealArgs& a) {
    if (a.fmode) {
        if (one) k_real_list<R, true, true><<<a.nlblk, kBlockP, 0, st>>>(a);
        else k_real_list<R, false, true><<<a.nlblk, kBlockP, 0, st>>>(a);
    } else {
        if (one) k_real_list<R, true, false><<<a.nlblk, kBlockP, 0, st>>>(a);
        else k_real_list<R, false, false><<<a.nlblk, kBlockP, 0, st>>>(a);
    }
}

void launch_real_list(cudaStream_t st, bool one, const RealArgs& a) {
    if (a.nlblk <= 0) return;
    switch (a.lsplit) {
        case 2: real_list_r<2>(st, one, a); break;
        case 4: real_list_r<4>(st, one, a); break;
        case 8: real_list_r<8>(st, one, a); break;
        default: real_list_r<1>(st, one, a); break;
    }
}

void launch_list_build(cudaStream_t st, bool one, const ListArgs& la) {
    if (la.nblk <= 0) return;
    if (one) k_list_build<true><<<la.nblk, kBlockP, 0, st>>>(la);
    else k_list_build<false><<<la.nblk, kBlockP, 0, st>>>(la);
}

void launch_real_f64(cudaStream_t st, bool one, const RealArgs& a) {
    if (a.nrblk <= 0) return;
    switch (a.split64) {
        case 2: real_f64_g<2>(st, one, a); break;
        case 4: real_f64_g<4>(st, one, a); break;
        case 8: real_f64_g<8>(st, one, a); break;
        case 16: real_f64_g<16>(st, one, a); break;
        case 32: real_f64_g<32>(st, one, a); break;
        default: real_f64_g<1>(st, one, a); break;
    }
}

void launch_energy(cudaStream_t st, bool one, const Work& w, int nsys, const int4* ksamp,
                   const unsigned long long* rho_fx, const double2* blk_e,
                   const double2* blk_q, const double2* blk_w, int parts, int per_cell,
                   double* E_out, double* W_out) {
    if (nsys <= 0) return;
    if (one)
        k_energy<true><<<nsys, 256, 0, st>>>(w, ksamp, rho_fx, blk_e, blk_q, blk_w, parts,
                                             per_cell, E_out, W_out);
    else
        k_energy<false><<<nsys, 256, 0, st>>>(w, ksamp, rho_fx, blk_e, blk_q, blk_w, parts,
                                              per_cell, E_out, W_out);
}

}  // namespace rbe
