// kbest_kernels.cu -- sm_103a kernels of the K-Best GED path.
//
//   pack_kernel   S0: edge lists -> adjacency bitsets and edge-label bit-planes
//   kbest_kernel  S1-S5 for every pair of a size class: persistent teams pull pairs from a
//                 device work queue; per level they stage the vertex-cost row, build per-node
//                 neighbour bitsets, score every successor with AND/XOR + popcount, select the
//                 best K with a deterministic stable counting sort, write the kept children in
//                 key order, and finally complete the leaves and take the argmin.
//
// Method: Algorithm 1 of Dabah & Herten (branching Sec. 4.1.1, evaluation Sec. 4.1.2 and
// Algorithm 2, selection Sec. 4.2, leaf insertions Sec. 4.4). The paper's GPU design
// (one block per node, a lambda walk per successor, atomic top-L lists) is replaced here:
// the implied edge cost of substituting v_i by u is computed from bitsets,
//     P     = images of the already-substituted g1 neighbours of v_i,
//     Img   = images of every substituted g1 vertex,
//     A2[u] = neighbours of u in g2,
//   inserted edges   = popc(A2[u] & Img & ~P)
//   deleted edges    = popc(P & ~A2[u]) + (# g1 neighbours of v_i that were deleted)
//   relabelled edges = popc(A2[u] & P & OR_b(PL_b ^ L2_b[u]))
// and when insertion and deletion cost the same, the first two fold into one
// popc((A2[u] & Img) ^ P) since P is a subset of Img.
#include <climits>
#include <cstdint>

#include "fastged_internal.h"

namespace fastged {

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// bits k of word w with k < i
__device__ __forceinline__ uint64_t low_mask(int i, int w)
{
    const int lo = w * 64;
    if (i >= lo + 64) return ~0ull;
    if (i <= lo) return 0ull;
    return (1ull << (i - lo)) - 1ull;
}

// ------------------------------------------------------------------------------------
// S0: pack edge lists into bitsets (one warp per graph, lanes over its edges).
// ------------------------------------------------------------------------------------
__global__ void pack_kernel(const PackParams pp)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g < pp.n_graphs; g += nwarps) {
        const GraphMeta mt = pp.gmeta[g];
        uint64_t *A = pp.adj + mt.adj_off;
        for (int k = lane; k < mt.m; k += 32) {
            const int64_t e = mt.edge_off + k;
            const int u = pp.edges[2 * e], v = pp.edges[2 * e + 1];
            const unsigned long long bu = 1ull << (u & 63), bv = 1ull << (v & 63);
            const unsigned long long old =
                atomicOr((unsigned long long *)&A[(int64_t)u * mt.W + (v >> 6)], bv);
            if (old & bv) atomicOr(pp.err, kErrDuplicateEdge);
            atomicOr((unsigned long long *)&A[(int64_t)v * mt.W + (u >> 6)], bu);
            if (pp.elabel) {
                const int lab = pp.elabel[e];
                for (int b = 0; b < pp.B; ++b) {
                    if (!((lab >> b) & 1)) continue;
                    uint64_t *Pl = pp.planes + mt.plane_off + (int64_t)b * mt.n * mt.W;
                    atomicOr((unsigned long long *)&Pl[(int64_t)u * mt.W + (v >> 6)], bv);
                    atomicOr((unsigned long long *)&Pl[(int64_t)v * mt.W + (u >> 6)], bu);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// K-Best teams
// ------------------------------------------------------------------------------------
struct TeamShared {
    int pair;
    int newL;
    int fast;
    int pbase;
    int delcost;
    int cnt;
    int mx;
    int maxb;     // largest histogram bucket touched at this level
    int thr;      // bucket holding the K-th smallest PED (fast path)
    int wmaxb[kMaxWarps];
    int wlt[kMaxWarps];
    int weq[kMaxWarps];
    unsigned long long wbest[kMaxWarps];
};

template <int W, typename MapT>
struct Regions {
    int32_t *hist, *bbase, *crow, *alpha2, *sbase, *sel, *selped, *tmp, *cand;
    int32_t *ped0, *ped1;
    uint64_t *a2t, *l2t, *img0, *img1, *P, *PL;
    uint8_t *map0, *map1;
};

// A kept child is stored in the selection list as (parent slot << 11) | j, j = 0..n2.
constexpr int kSelShift = 11;

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: cycles thread 0 of every team spends in each phase
__device__ unsigned long long g_phase_cycles[8];
#define PHASE_MARK(k)                                        \
    do {                                                     \
        if (threadIdx.x == 0) {                              \
            const long long t_ = clock64();                  \
            ph[k] += t_ - ph_last;                           \
            ph_last = t_;                                    \
        }                                                    \
    } while (0)
#else
#define PHASE_MARK(k) do { } while (0)
#endif

// Exact fallback of the selection when the kept set reaches past the histogram window:
// the K-th smallest PED is found by bisection over block-wide counts, the kept candidates
// are compacted stably in enumeration order, then ranked by (PED, enumeration index).
template <int W, typename MapT>
__device__ __forceinline__ void select_exact(const Regions<W, MapT> R, TeamShared &S, int L,
                                             int stride, int newL, int lo)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = blockDim.x, NW = T >> 5;
    const int N = L * stride;

    // largest valid PED
    int mx = 0;
    for (int c = tid; c < N; c += T) {
        const int v = R.cand[c];
        if (v != INT_MAX && v > mx) mx = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) S.mx = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&S.mx, mx);
    __syncthreads();
    int hi = S.mx;
    if (lo > hi) lo = hi;
    // invariant: count(PED < lo) < newL <= count(PED <= hi)
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        int cnt = 0;
        for (int c = tid; c < N; c += T) cnt += (R.cand[c] <= mid);
        cnt = warp_sum(cnt);
        __syncthreads();
        if (tid == 0) S.cnt = 0;
        __syncthreads();
        if (lane == 0) atomicAdd(&S.cnt, cnt);
        __syncthreads();
        if (S.cnt >= newL) hi = mid; else lo = mid + 1;
    }
    const int thr = lo;

    // per-warp counts of PED < thr and PED == thr over the warp's contiguous slot range
    const int s_lo = (warp * L) / NW, s_hi = ((warp + 1) * L) / NW;
    const int c_lo = s_lo * stride, c_hi = s_hi * stride;
    int nlt = 0, neq = 0;
    for (int cb = c_lo; cb < c_hi; cb += 32) {
        const int cc = cb + lane;
        const int v = cc < c_hi ? R.cand[cc] : INT_MAX;
        nlt += __popc(__ballot_sync(0xffffffffu, v < thr));
        neq += __popc(__ballot_sync(0xffffffffu, v == thr));
    }
    if (lane == 0) { S.wlt[warp] = nlt; S.weq[warp] = neq; }
    __syncthreads();
    int lt_all = 0;
    for (int w = 0; w < NW; ++w) lt_all += S.wlt[w];
    const int q = newL - lt_all;   // ties at thr that are kept, first in enumeration order
    int keep_before = 0, eq_before = 0;
    for (int w = 0; w < warp; ++w) {
        const int take = min(max(q - eq_before, 0), S.weq[w]);
        keep_before += S.wlt[w] + take;
        eq_before += S.weq[w];
    }
    for (int cb = c_lo; cb < c_hi; cb += 32) {
        const int cc = cb + lane;
        const int v = cc < c_hi ? R.cand[cc] : INT_MAX;
        const bool is_eq = (v == thr);
        const unsigned eqb = __ballot_sync(0xffffffffu, is_eq);
        const int eq_rank = eq_before + __popc(eqb & lanemask_lt());
        const bool keep = (v < thr) || (is_eq && eq_rank < q);
        const unsigned kb = __ballot_sync(0xffffffffu, keep);
        if (keep) R.tmp[keep_before + __popc(kb & lanemask_lt())] = cc;
        keep_before += __popc(kb);
        eq_before += __popc(eqb);
    }
    __syncthreads();
    // rank by (PED, enumeration index); tmp is already in enumeration order
    for (int a = tid; a < newL; a += T) {
        const int ca = R.tmp[a];
        const int pa = R.cand[ca];
        int rank = 0;
        for (int b = 0; b < newL; ++b) {
            const int pb = R.cand[R.tmp[b]];
            rank += (pb < pa) || (pb == pa && b < a);
        }
        const int s = ca / stride;
        R.sel[rank] = (s << kSelShift) | (ca - s * stride);
        R.selped[rank] = pa;
    }
}

template <int W, typename MapT>
__device__ __forceinline__ void solve_pair(const KParams &p, const Regions<W, MapT> R,
                                           TeamShared &S, const int pair)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = blockDim.x, NW = T >> 5;
    const int g1 = p.pairs[2 * pair], g2 = p.pairs[2 * pair + 1];
    const GraphMeta m1 = p.gmeta[g1], m2 = p.gmeta[g2];
    const int n1 = m1.n, n2 = m2.n, W1 = m1.W, W2 = m2.W;
    const int K = p.kpp ? p.kpp[pair] : p.K;
    const int B = p.lay.B;
    const int N2S = p.lay.n2s;
    const int KM = p.lay.kmax;
    const int64_t mrow = p.lay.mrow;
    const int stride = n2 + 1;
    const MapT DEL = (MapT)~(MapT)0;
    const CostModel c = p.cost;
    const int hwin = p.hwin;
    const bool fold_ie = (c.eins == c.edel);
    // small bitsets keep the target vertex's rows in registers for a whole level
    constexpr bool HOIST = (W <= 2);
    constexpr int HW = HOIST ? W : 1;
#ifdef FASTGED_PHASE_TIMERS
    long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long ph_last = clock64();
#endif

    // stage g2: transposed adjacency and label planes, vertex labels; clear the histogram
    {
        const uint64_t *adj2 = p.adj + m2.adj_off;
        for (int idx = tid; idx < W * n2; idx += T) {
            const int w = idx / n2, u = idx - w * n2;
            R.a2t[w * N2S + u] = (w < W2) ? adj2[(int64_t)u * W2 + w] : 0ull;
        }
        for (int b = 0; b < B; ++b) {
            const uint64_t *pl2 = p.planes + m2.plane_off + (int64_t)b * n2 * W2;
            for (int idx = tid; idx < W * n2; idx += T) {
                const int w = idx / n2, u = idx - w * n2;
                R.l2t[(b * W + w) * N2S + u] = (w < W2) ? pl2[(int64_t)u * W2 + w] : 0ull;
            }
        }
        for (int u = tid; u < n2; u += T) R.alpha2[u] = p.vlab[m2.lab_off + u];
        for (int x = tid; x < hwin * NW; x += T) R.hist[x] = 0;
        // root node: empty lambda, R_V2 = V2, PED 0
        for (int w = tid; w < W; w += T) R.img0[w] = 0ull;
        if (tid == 0) {
            R.ped0[0] = 0;
            S.maxb = -1;
        }
    }
    long long nevals = 0;
    int L = 1;
    // current / next beam buffers, swapped after every level
    uint8_t *mapc = R.map0, *mapn = R.map1;
    uint64_t *imgc = R.img0, *imgn = R.img1;
    int32_t *pedc = R.ped0, *pedn = R.ped1;
    __syncthreads();
    PHASE_MARK(0);

    for (int i = 0; i < n1; ++i) {
        // ---- S1 cost row + S2 per-node vectors -------------------------------------
        const uint64_t *row1 = p.adj + m1.adj_off + (int64_t)i * W1;
        const uint64_t *pl1 = p.planes + m1.plane_off + (int64_t)i * W1;
        const int64_t pl1_step = (int64_t)n1 * W1;
        {
            const int a1 = p.vlab[m1.lab_off + i];
            for (int j = tid; j < n2; j += T) R.crow[j] = (R.alpha2[j] != a1) ? c.vsub : 0;
            // clear the buckets the previous level touched
            for (int x = tid; x < (S.maxb + 1) * NW; x += T) R.hist[x] = 0;
            for (int s = tid; s < L; s += T) {
                uint64_t *Ps = R.P + (int64_t)s * W;
#pragma unroll
                for (int w = 0; w < W; ++w) Ps[w] = 0ull;
                for (int b = 0; b < B; ++b)
                    for (int w = 0; w < W; ++w) R.PL[((int64_t)b * KM + s) * W + w] = 0ull;
                const MapT *ms = (const MapT *)(mapc + (int64_t)s * mrow);
                int dcnt = 0;
                for (int w = 0; w < W1; ++w) {
                    uint64_t bits = row1[w] & low_mask(i, w);
                    while (bits) {
                        const int t = __ffsll((long long)bits) - 1;
                        bits &= bits - 1ull;
                        const MapT phi = ms[w * 64 + t];
                        if (phi == DEL) { ++dcnt; continue; }
                        const int pw = (int)phi >> 6;
                        const uint64_t pb = 1ull << ((int)phi & 63);
                        Ps[pw] |= pb;
                        for (int b = 0; b < B; ++b)
                            if ((pl1[b * pl1_step + w] >> t) & 1ull)
                                R.PL[((int64_t)b * KM + s) * W + pw] |= pb;
                    }
                }
                R.sbase[s] = pedc[s] + c.edel * dcnt;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int d = 0;
            for (int w = 0; w < W1; ++w) d += __popcll(row1[w] & low_mask(i, w));
            S.delcost = c.vdel + c.edel * d;   // v_i -> eps takes its edges to v_0..v_{i-1}
            S.pbase = pedc[0];                 // kept list is sorted: slot 0 has the least PED
        }
        __syncthreads();
        PHASE_MARK(1);

        // ---- S3 successor evaluation + per-warp PED histogram -----------------------
        // lane <-> target vertex u_j (j = jb + lane); the warp walks its contiguous slots
        const int pbase = S.pbase, delcost = S.delcost;
        const int s_lo = (warp * L) / NW, s_hi = ((warp + 1) * L) / NW;
        int32_t *hcol = R.hist + warp;
        int wmaxb = -1;
        for (int jb = 0; jb < stride; jb += 32) {
            const int j = jb + lane;
            const bool is_sub = j < n2, is_del = (j == n2);
            uint64_t a[HW], l0[HW], l1[HW];
            int cj = 0;
#pragma unroll
            for (int w = 0; w < HW; ++w) { a[w] = 0ull; l0[w] = 0ull; l1[w] = 0ull; }
            if (is_sub) {
                cj = R.crow[j];
                if (HOIST) {
#pragma unroll
                    for (int w = 0; w < HW; ++w) {
                        a[w] = R.a2t[w * N2S + j];
                        if (B > 0) l0[w] = R.l2t[(0 * W + w) * N2S + j];
                        if (B > 1) l1[w] = R.l2t[(1 * W + w) * N2S + j];
                    }
                }
            }
            const uint64_t jbit = 1ull << (j & 63);
            const int jw = j >> 6;
            for (int s = s_lo; s < s_hi; ++s) {
                int ped = INT_MAX;
                if (is_del) {
                    ped = pedc[s] + delcost;
                } else if (is_sub) {
                    const uint64_t *im = imgc + (int64_t)s * W;
                    if (!(im[jw] & jbit)) {
                        const uint64_t *Ps = R.P + (int64_t)s * W;
                        int x = 0, y = 0, z = 0;
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            const uint64_t aw = HOIST ? a[HOIST ? w : 0] : R.a2t[w * N2S + j];
                            const uint64_t ai = aw & im[w];
                            const uint64_t pw = Ps[w];
                            if (fold_ie) {
                                x += __popcll(ai ^ pw);
                            } else {
                                x += __popcll(ai & ~pw);
                                y += __popcll(pw & ~aw);
                            }
                            if (B > 0) {
                                uint64_t ld;
                                if (HOIST && B <= 2) {
                                    ld = R.PL[((int64_t)0 * KM + s) * W + w] ^ l0[HOIST ? w : 0];
                                    if (B > 1)
                                        ld |= R.PL[((int64_t)1 * KM + s) * W + w] ^ l1[HOIST ? w : 0];
                                } else {
                                    ld = 0ull;
                                    for (int b = 0; b < B; ++b)
                                        ld |= R.PL[((int64_t)b * KM + s) * W + w] ^
                                              R.l2t[(b * W + w) * N2S + j];
                                }
                                z += __popcll(aw & pw & ld);
                            }
                        }
                        ped = R.sbase[s] + cj + c.eins * x + c.edel * y + c.esub * z;
                    }
                }
                if (j < stride) R.cand[s * stride + j] = ped;
                int bkt = -1;
                if (ped != INT_MAX) {
                    const int d = ped - pbase;
                    bkt = d < hwin - 1 ? d : hwin - 1;
                    wmaxb = bkt > wmaxb ? bkt : wmaxb;
                }
                const unsigned mm = __match_any_sync(0xffffffffu, bkt);
                if (bkt >= 0 && lane == __ffs(mm) - 1) hcol[bkt * NW] += __popc(mm);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmaxb = max(wmaxb, __shfl_xor_sync(0xffffffffu, wmaxb, o));
        if (lane == 0) S.wmaxb[warp] = wmaxb;
        __syncthreads();
        PHASE_MARK(2);

        // ---- S4 selection: scan of the (bucket, warp) histogram ---------------------
        int maxb = -1;
        for (int w = 0; w < NW; ++w) maxb = max(maxb, S.wmaxb[w]);
        const int nb = maxb + 1;   // >= 1: every node has a deletion child
        for (int b = tid; b < nb; b += T) {
            int run = 0;
            for (int w = 0; w < NW; ++w) {
                const int v = R.hist[b * NW + w];
                R.hist[b * NW + w] = run;
                run += v;
            }
            R.bbase[b] = run;
        }
        __syncthreads();
        if (warp == 0) {
            const int per = (nb + 31) >> 5;
            int loc = 0;
            for (int k = 0; k < per; ++k) {
                const int b = lane * per + k;
                if (b < nb) loc += R.bbase[b];
            }
            int incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int nl = min(K, total);
            int run = incl - loc;
            for (int k = 0; k < per; ++k) {
                const int b = lane * per + k;
                if (b < nb) {
                    const int v = R.bbase[b];
                    R.bbase[b] = run;
                    if (run < nl && run + v >= nl) S.thr = b;   // exactly one bucket crosses
                    run += v;
                }
            }
            if (lane == 0) {
                S.newL = nl;
                S.maxb = maxb;
                nevals += total;
            }
        }
        __syncthreads();
        const int newL = S.newL;
        const int thr = S.thr;
        if (thr < hwin - 1) {
            // stable counting sort restricted to buckets <= thr: position = #(smaller PED)
            // + #(equal PED earlier in (slot, j) order)
            for (int s = s_lo; s < s_hi; ++s) {
                for (int jb = 0; jb < stride; jb += 32) {
                    const int j = jb + lane;
                    const int ped = j < stride ? R.cand[s * stride + j] : INT_MAX;
                    int bkt = -1;
                    if (ped != INT_MAX && ped - pbase <= thr) bkt = ped - pbase;
                    if (__ballot_sync(0xffffffffu, bkt >= 0) == 0u) continue;
                    const unsigned mm = __match_any_sync(0xffffffffu, bkt);
                    if (bkt >= 0) {
                        const int pos = R.bbase[bkt] + hcol[bkt * NW] + __popc(mm & lanemask_lt());
                        if (pos < newL) {
                            R.sel[pos] = (s << kSelShift) | j;
                            R.selped[pos] = ped;
                        }
                    }
                    __syncwarp();
                    if (bkt >= 0 && lane == __ffs(mm) - 1) hcol[bkt * NW] += __popc(mm);
                    __syncwarp();
                }
            }
        } else {
            select_exact<W, MapT>(R, S, L, stride, newL, pbase + hwin - 1);
        }
        __syncthreads();
        PHASE_MARK(3);

        // ---- kept children, in key order (slot = rank) -----------------------------
        {
            const int nvec = (int)((i * (int)sizeof(MapT) + 15) >> 4);
            if (mrow <= 128) {
                for (int r = tid; r < newL; r += T) {
                    const int v = R.sel[r];
                    const int s = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                    const uint4 *src = (const uint4 *)(mapc + (int64_t)s * mrow);
                    uint4 *dst = (uint4 *)(mapn + (int64_t)r * mrow);
                    for (int t = 0; t < nvec; ++t) dst[t] = src[t];
                    ((MapT *)dst)[i] = (j < n2) ? (MapT)j : DEL;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        uint64_t x = imgc[(int64_t)s * W + w];
                        if (j < n2 && (j >> 6) == w) x |= 1ull << (j & 63);
                        imgn[(int64_t)r * W + w] = x;
                    }
                    pedn[r] = R.selped[r];
                }
            } else {
                for (int r = warp; r < newL; r += NW) {
                    const int v = R.sel[r];
                    const int s = v >> kSelShift, j = v & ((1 << kSelShift) - 1);
                    const uint4 *src = (const uint4 *)(mapc + (int64_t)s * mrow);
                    uint4 *dst = (uint4 *)(mapn + (int64_t)r * mrow);
                    for (int t = lane; t < nvec; t += 32) dst[t] = src[t];
                    for (int w = lane; w < W; w += 32) {
                        uint64_t x = imgc[(int64_t)s * W + w];
                        if (j < n2 && (j >> 6) == w) x |= 1ull << (j & 63);
                        imgn[(int64_t)r * W + w] = x;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        ((MapT *)dst)[i] = (j < n2) ? (MapT)j : DEL;
                        pedn[r] = R.selped[r];
                    }
                }
            }
        }
        __syncthreads();
        PHASE_MARK(4);
        { uint8_t *t = mapc; mapc = mapn; mapn = t; }
        { uint64_t *t = imgc; imgc = imgn; imgn = t; }
        { int32_t *t = pedc; pedc = pedn; pedn = t; }
        L = newL;
    }

    // ---- S5 leaf completion (insert the free g2 vertices and their edges) + argmin ------
    {
        unsigned long long best = ~0ull;
        for (int s = warp; s < L; s += NW) {
            const uint64_t *im = imgc + (int64_t)s * W;
            int acc = 0;
            for (int u = lane; u < n2; u += 32) {
                if ((im[u >> 6] >> (u & 63)) & 1ull) {
#pragma unroll
                    for (int w = 0; w < W; ++w) acc += __popcll(R.a2t[w * N2S + u] & im[w]);
                }
            }
            int nimg = 0;
            for (int w = lane; w < W; w += 32) nimg += __popcll(im[w]);
            acc = warp_sum(acc);
            nimg = warp_sum(nimg);
            // g2 edges with both ends used were counted twice in acc
            const long long total = (long long)pedc[s] + (long long)c.vins * (n2 - nimg) +
                                    (long long)c.eins * (m2.m - acc / 2);
            const unsigned long long key = ((unsigned long long)total << 32) | (unsigned)s;
            best = key < best ? key : best;
        }
        if (lane == 0) S.wbest[warp] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = S.wbest[0];
            for (int w = 1; w < NW; ++w) b = S.wbest[w] < b ? S.wbest[w] : b;
            S.wbest[0] = b;
            p.out_cost[pair] = (int32_t)(b >> 32);
            if (p.out_nevals) p.out_nevals[pair] = nevals + L;
        }
        __syncthreads();
        const int bs = (int)(S.wbest[0] & 0xffffffffull);
        const MapT *mb = (const MapT *)(mapc + (int64_t)bs * mrow);
        int32_t *om = p.out_map + p.map_off[pair];
        for (int k = tid; k < n1; k += T) {
            const MapT v = mb[k];
            om[k] = (v == DEL) ? -1 : (int32_t)v;
        }
        __syncthreads();
        PHASE_MARK(5);
    }
#ifdef FASTGED_PHASE_TIMERS
    if (tid == 0)
        for (int k = 0; k < 6; ++k) atomicAdd(&g_phase_cycles[k], (unsigned long long)ph[k]);
#endif
}

template <int W, typename MapT>
__global__ void __launch_bounds__(512, 2) kbest_kernel(const KParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ TeamShared S;
    uint8_t *gs = p.gscratch + (int64_t)blockIdx.x * p.lay.slice_bytes;
    auto base = [&](int r) -> uint8_t * {
        return ((p.lay.smem_mask >> r) & 1u ? smem : gs) + p.lay.off[r];
    };
    Regions<W, MapT> R;
    R.hist = (int32_t *)base(RG_HIST);
    R.bbase = (int32_t *)base(RG_BBASE);
    R.crow = (int32_t *)base(RG_CROW);
    R.alpha2 = (int32_t *)base(RG_ALPHA2);
    R.a2t = (uint64_t *)base(RG_A2T);
    R.l2t = (uint64_t *)base(RG_L2T);
    R.sbase = (int32_t *)base(RG_SBASE);
    R.ped0 = (int32_t *)base(RG_PED0);
    R.ped1 = (int32_t *)base(RG_PED1);
    R.sel = (int32_t *)base(RG_SEL);
    R.selped = (int32_t *)base(RG_SELPED);
    R.img0 = (uint64_t *)base(RG_IMG0);
    R.img1 = (uint64_t *)base(RG_IMG1);
    R.P = (uint64_t *)base(RG_P);
    R.PL = (uint64_t *)base(RG_PL);
    R.cand = (int32_t *)base(RG_CAND);
    R.map0 = base(RG_MAP0);
    R.map1 = base(RG_MAP1);
    R.tmp = (int32_t *)base(RG_TMP);

    for (;;) {
        if (threadIdx.x == 0) S.pair = atomicAdd(p.queue_head, 1);
        __syncthreads();
        const int qi = S.pair;
        __syncthreads();
        if (qi >= p.n_order) break;
        solve_pair<W, MapT>(p, R, S, p.order[qi]);
    }
}

// ------------------------------------------------------------------------------------
// launch wrappers (host side of this translation unit)
// ------------------------------------------------------------------------------------
// Opts the kernel into the device's full dynamic shared memory (needed above 48 KB) before
// it is launched or queried for occupancy.
template <int W, typename MapT>
static cudaError_t ensure_smem_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kbest_kernel<W, MapT>);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kbest_kernel<W, MapT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int W, typename MapT>
static cudaError_t launch_one(const KParams &p, int grid, int block, size_t smem,
                              cudaStream_t st)
{
    cudaError_t e = ensure_smem_attr<W, MapT>();
    if (e != cudaSuccess) return e;
    kbest_kernel<W, MapT><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int W, typename MapT>
static cudaError_t occupancy_one(int block, size_t smem, int *out)
{
    cudaError_t e = ensure_smem_attr<W, MapT>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kbest_kernel<W, MapT>, block, smem);
}

#define FASTGED_DISPATCH(W_, wide, CALL)                                          \
    do {                                                                          \
        switch (W_) {                                                             \
        case 1: if (wide) return CALL(1, uint16_t); else return CALL(1, uint8_t); \
        case 2: if (wide) return CALL(2, uint16_t); else return CALL(2, uint8_t); \
        case 4: if (wide) return CALL(4, uint16_t); else return CALL(4, uint8_t); \
        case 8: return CALL(8, uint16_t);                                         \
        case 16: return CALL(16, uint16_t);                                       \
        default: return cudaErrorInvalidValue;                                    \
        }                                                                         \
    } while (0)

cudaError_t launch_kbest(int W, bool wide_map, const KParams &p, int grid, int block,
                         size_t smem, cudaStream_t st)
{
#define CALL_LAUNCH(w, M) launch_one<w, M>(p, grid, block, smem, st)
    FASTGED_DISPATCH(W, wide_map, CALL_LAUNCH);
#undef CALL_LAUNCH
}

cudaError_t kbest_occupancy(int W, bool wide_map, int block, size_t smem, int *out)
{
#define CALL_OCC(w, M) occupancy_one<w, M>(block, smem, out)
    FASTGED_DISPATCH(W, wide_map, CALL_OCC);
#undef CALL_OCC
}

cudaError_t launch_pack(const PackParams &pp, int n_graphs, cudaStream_t st)
{
    const int block = 256;
    int grid = (n_graphs * 32 + block - 1) / block;
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    pack_kernel<<<grid, block, 0, st>>>(pp);
    return cudaGetLastError();
}

// upper bound of the kernels' static shared memory (the team's scalars)
size_t team_shared_static_bytes() { return sizeof(TeamShared) + 256; }

}  // namespace fastged

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: reads (and optionally clears) the per-phase cycle counters
extern "C" int fastged_debug_phase_cycles(unsigned long long *out, int reset)
{
    if (cudaMemcpyFromSymbol(out, fastged::g_phase_cycles, sizeof(unsigned long long) * 8) !=
        cudaSuccess)
        return -3;
    if (reset) {
        unsigned long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        cudaMemcpyToSymbol(fastged::g_phase_cycles, z, sizeof(z));
    }
    return 0;
}
#endif
