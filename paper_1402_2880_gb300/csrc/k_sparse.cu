// Sparse products of the C^T X C kernel (Section "Computation kernel for the
// matrix products C^T X C") and the density / Mulliken charges (Eq. pop).
//
// The paper builds C^T X C from 16-column strips of X C computed with dense
// 16x16 blocks. Here the 16-column strip is a tile: Y = X C is formed per
// tile column (column-major, only the row blocks reachable through X), and
// every kept block of C^T X C is one output-stationary 16x16 tile pair
// reduced over the row blocks the two columns share.
#include "sscf_internal.h"

#include <type_traits>

namespace sscf {

namespace {

template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

// ---------------------------------------------------------------------------
// Column index of C: per tile, the (row block, slot) pairs sorted by row.
// ---------------------------------------------------------------------------
__global__ void k_ci_count(int n_mol, int cap, const int* __restrict__ c_nt, const int* __restrict__ c_tile,
                           int* __restrict__ cnt) {
    int r = blockIdx.x;
    for (int s = threadIdx.x; s < c_nt[r]; s += blockDim.x) atomicAdd(&cnt[c_tile[(size_t)r * cap + s]], 1);
}

// exclusive scan of n counts into ptr (n + 1 entries); one CTA of 1024 threads
__global__ void k_scan(int n, const int* __restrict__ cnt, int* __restrict__ ptr) {
    __shared__ int part[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            int v = part[i];
            part[i] = run;
            run += v;
        }
        ptr[n] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int i = lo; i < hi; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
}

__global__ void k_ci_fill(int n_mol, int cap, const int* __restrict__ c_nt, const int* __restrict__ c_tile,
                          const int* __restrict__ ptr, int* __restrict__ cursor, int* __restrict__ row,
                          int* __restrict__ slot) {
    int r = blockIdx.x;
    for (int s = threadIdx.x; s < c_nt[r]; s += blockDim.x) {
        int t = c_tile[(size_t)r * cap + s];
        int pos = ptr[t] + atomicAdd(&cursor[t], 1);
        row[pos] = r;
        slot[pos] = s;
    }
}

// Sort every tile's segment by row. The rows of one tile are distinct and lie
// in its cluster, so a bitmap over the cluster's rows orders them: an entry
// moves to the number of set bits below its row. One CTA per tile.
constexpr int kSortMax = 8192;          // entries per tile (16 per thread)
constexpr int kSortThreads = 512;
__global__ void __launch_bounds__(kSortThreads) k_ci_sort(const int* __restrict__ ptr, int* __restrict__ row,
                                                          int* __restrict__ slot, const int* __restrict__ tile_row0,
                                                          int n_rows, unsigned* __restrict__ err) {
    extern __shared__ unsigned sbits[];               // n_rows bits, then the set bits before each word
    const int nw = (n_rows + 31) >> 5;
    int* wpre = (int*)(sbits + nw);
    __shared__ int part[kSortThreads];
    const int t = blockIdx.x;
    const int lo = ptr[t], n = ptr[t + 1] - lo;
    if (n <= 1) return;
    if (n > kSortMax) {
        if (threadIdx.x == 0) atomicOr(err, kErrSortSize);
        return;
    }
    const int r0 = tile_row0[t];
    for (int w = threadIdx.x; w < nw; w += blockDim.x) sbits[w] = 0u;
    __syncthreads();
    constexpr int kPer = kSortMax / kSortThreads;
    int rv[kPer], sv[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = threadIdx.x + j * kSortThreads;
        if (i < n) {
            rv[j] = row[lo + i];
            sv[j] = slot[lo + i];
            const int rr = rv[j] - r0;
            atomicOr(&sbits[rr >> 5], 1u << (rr & 31));
        }
    }
    __syncthreads();
    const int per = (nw + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(nw, w0 + per);
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(sbits[w]);
    part[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int w = w0; w < w1; ++w) {
        wpre[w] = run;
        run += __popc(sbits[w]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = threadIdx.x + j * kSortThreads;
        if (i < n) {
            const int rr = rv[j] - r0;
            const int pos = wpre[rr >> 5] + __popc(sbits[rr >> 5] & ((1u << (rr & 31)) - 1u));
            row[lo + pos] = rv[j];
            slot[lo + pos] = sv[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Y[:, t] = X C[:, t] for tiles t in [tile_lo, tile_hi), column-major output.
// One CTA per tile: mark the row blocks reachable from the tile's rows
// through the molecule-pair pattern (tiles below own_below: the tile's own
// rows only), then one warp per output row block sums X[r, n] (6x6)
// C[n, t] (6x16) over the pattern neighbours n holding t.
// ---------------------------------------------------------------------------
constexpr int kXcBatch = 4;   // matched neighbours whose loads are in flight together
template <typename T>
__global__ void k_xc(int tile_lo, int n_rows, int own_below, int cap, int capY, const int* __restrict__ tile_row0,
                     const int* __restrict__ cci_ptr, const int* __restrict__ cci_row,
                     const int* __restrict__ cci_slot, const T* __restrict__ c_val, const int* __restrict__ mp_ptr,
                     const int* __restrict__ mp_col, const T* __restrict__ Xb, int* __restrict__ y_n,
                     int* __restrict__ y_row, T* __restrict__ y_val, unsigned* __restrict__ err) {
    // row maps are local to the tile's cluster: row r -> r - r0, n_rows = largest cluster
    extern __shared__ int sm[];
    const int nw = (n_rows + 31) / 32;
    unsigned* bits = (unsigned*)sm;               // n_rows bits
    int* wpre = (int*)(bits + nw);                // prefix of popcounts per word
    short* rowpos = (short*)(wpre + nw);          // n_rows: index into the tile's column list or -1
    __shared__ int s_total;
    // tiles from own_below on (the longer ones: every reachable row) first
    const int t = tile_lo + (int)((blockIdx.x + (unsigned)max(own_below - tile_lo, 0)) % gridDim.x);
    const int r0 = tile_row0[t];
    const int lo = cci_ptr[t], nc = cci_ptr[t + 1] - lo;
    if (nc > 32767) {   // the 16-bit row map cannot index this column
        if (threadIdx.x == 0) {
            atomicOr(err, kErrCapacity);
            y_n[t] = 0;
        }
        return;
    }
    for (int i = threadIdx.x; i < n_rows; i += blockDim.x) rowpos[i] = -1;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) bits[i] = 0u;
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) rowpos[cci_row[lo + k] - r0] = (short)k;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        int r = cci_row[lo + k];
        if (t < own_below) {   // Y only where C[:, t] has rows: enough for C[:, t]^T Y[:, t]
            const int n = r - r0;
            atomicOr(&bits[n >> 5], 1u << (n & 31));
            continue;
        }
        for (int e = mp_ptr[r]; e < mp_ptr[r + 1]; ++e) {
            int n = mp_col[e] - r0;
            atomicOr(&bits[n >> 5], 1u << (n & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < nw; ++w) {
            wpre[w] = run;
            run += __popc(bits[w]);
        }
        s_total = run;
    }
    __syncthreads();
    const int ny = s_total;
    if (ny > capY) {
        if (threadIdx.x == 0) {
            atomicOr(err, kErrCapacity);
            y_n[t] = 0;
        }
        return;
    }
    if (threadIdx.x == 0) y_n[t] = ny;
    // write sorted row list
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        unsigned b = bits[w];
        int p = wpre[w];
        while (b) {
            int i = __ffs(b) - 1;
            b &= b - 1;
            y_row[(size_t)t * capY + p++] = r0 + w * 32 + i;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int col = lane & 15, q0 = lane >> 4;   // AO rows q0, q0+2, q0+4
    using A = typename Acc<T>::type;
    for (int k = warp; k < ny; k += nwarps) {
        const int r = y_row[(size_t)t * capY + k];
        A acc0 = 0, acc1 = 0, acc2 = 0;
        // 32 pattern neighbours at a time: their ids, positions and slots are
        // looked up in parallel, one per lane; the matched ones are then summed
        // in pattern order with their data broadcast from the owning lane
        const int e_lo = mp_ptr[r], e_hi = mp_ptr[r + 1];
        for (int eb = e_lo; eb < e_hi; eb += 32) {
            const int e = eb + lane;
            int sl = -1, nl = 0;
            if (e < e_hi) {
                nl = mp_col[e];
                const int j = rowpos[nl - r0];
                if (j >= 0) sl = cci_slot[lo + j];
            }
            unsigned mm = __ballot_sync(0xffffffffu, sl >= 0);
            while (mm) {
                // kXcBatch matched neighbours per round: their loads in flight together, sums in order
                int src[kXcBatch];
#pragma unroll
                for (int u = 0; u < kXcBatch; ++u) {
                    src[u] = mm ? __ffs(mm) - 1 : -1;
                    if (mm) mm &= mm - 1;
                }
                A c6[kXcBatch][6];
                const T* xb[kXcBatch];
#pragma unroll
                for (int u = 0; u < kXcBatch; ++u) {
                    const int sv = src[u] < 0 ? 0 : src[u];
                    const int n = __shfl_sync(0xffffffffu, nl, sv);
                    const int ss = __shfl_sync(0xffffffffu, sl, sv);
                    xb[u] = Xb + (size_t)(eb + sv) * 36;
                    if (src[u] >= 0) {
                        const T* cv = c_val + ((size_t)n * cap + ss) * kTileVals + col;
#pragma unroll
                        for (int q = 0; q < 6; ++q) c6[u][q] = (A)cv[q * kTileW];
                    }
                }
#pragma unroll
                for (int u = 0; u < kXcBatch; ++u) {
                    if (src[u] < 0) continue;
                    // the lane's three rows of the 6x6 block, two values per load
                    // (rows start 6 values apart: 8-byte aligned for FP32, 16 for FP64)
                    using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
                    A xr[3][6];
#pragma unroll
                    for (int rr = 0; rr < 3; ++rr) {
                        const V2* x2 = (const V2*)(xb[u] + (q0 + 2 * rr) * 6);
#pragma unroll
                        for (int h = 0; h < 3; ++h) {
                            const V2 v = x2[h];
                            xr[rr][2 * h] = (A)v.x;
                            xr[rr][2 * h + 1] = (A)v.y;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        acc0 += xr[0][q] * c6[u][q];
                        acc1 += xr[1][q] * c6[u][q];
                        acc2 += xr[2][q] * c6[u][q];
                    }
                }
            }
        }
        T* yv = y_val + ((size_t)t * capY + k) * kTileVals;
        yv[(q0)*kTileW + col] = (T)acc0;
        yv[(q0 + 2) * kTileW + col] = (T)acc1;
        yv[(q0 + 4) * kTileW + col] = (T)acc2;
    }
}

// ---------------------------------------------------------------------------
// Tile-pair transform: out[p] (16x16) = C[:, a]^T Y[:, b] for every listed
// pair (a, b). One CTA per tile a with a shared map row block -> slot of a.
// One warp per pair: it walks b's rows (sorted), and for the rows present in
// a it stages the two 6x16 tiles (C[r, a] and Y[r, b]) in a per-warp buffer
// with 16-byte loads, kStage row blocks at a time; every lane then owns a 2x4
// block of the 16x16 result and does 8 FMAs per K step from one 8-byte and
// one 16-byte shared load. Rows are summed in ascending order (fixed order);
// mixed precision flushes the FP32 partial sums to FP64 every 32 rows.
// ---------------------------------------------------------------------------
constexpr int kTfWarps = 4;
constexpr int kStage = 4;   // row blocks staged per warp at a time
constexpr int kTcStride = 24;   // floats per staged AO row in the tensor-core path (bank-conflict-free fragments)
constexpr int kTcRows = kStage * kAoPerMol;   // staged AO rows (K) per round: 24 = 3 k-steps of 8

// x = hi + lo with hi, lo in TF32 (10 explicit mantissa bits each): hi by
// round-to-nearest, lo the rounded remainder, so hi + lo carries ~21 bits.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float r = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    hi = h;
    lo = l;
}

// D (16x8, FP32) += A (16x8, TF32, row-major) x B (8x8, TF32, column-major)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double2; };

// Staged values per warp: FP64 [kStage][2][96]; FP32 (tensor cores) C rows
// then Y rows, kTcRows rows of kTcStride floats each.
template <typename T> __host__ __device__ constexpr int tf_stage_vals() {
    return std::is_same<T, float>::value ? 2 * kTcRows * kTcStride : kStage * 2 * kTileVals;
}

// MINB: resident CTAs per SM the register budget is cut for (1: no cut)
template <typename T, int MINB>
__global__ void __launch_bounds__(kTfWarps * 32, MINB)
k_transform(int n_split, int n_rows, const int* __restrict__ tile_row0, int cap, int capY, const int* __restrict__ tp_ptr,
            const int* __restrict__ tp_b,
            const int* __restrict__ tp_out, const int* __restrict__ cci_ptr, const int* __restrict__ cci_row,
            const int* __restrict__ cci_slot, const T* __restrict__ c_val, const int* __restrict__ y_n,
            const int* __restrict__ y_row, const T* __restrict__ y_val, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sraw[];
    T* stage = (T*)sraw;                                        // [warps][tf_stage_vals]
    short* slot_of = (short*)(stage + (size_t)kTfWarps * tf_stage_vals<T>());   // n_rows (cluster-local)
    // CTA (a, s) takes the pairs of tile a with index = s (mod n_split)
    const int a = blockIdx.x / n_split, split = blockIdx.x % n_split;
    const int p0 = tp_ptr[a], p1 = tp_ptr[a + 1];
    if (p0 + split >= p1) return;
    const int r0 = tile_row0[a];
    const int lo = cci_ptr[a], nc = cci_ptr[a + 1] - lo;
    for (int i = threadIdx.x; i < n_rows; i += blockDim.x) slot_of[i] = -1;
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) slot_of[cci_row[lo + k] - r0] = (short)cci_slot[lo + k];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* buf = stage + (size_t)warp * tf_stage_vals<T>();
    if constexpr (std::is_same<T, float>::value) {
        // FP32 storage: the 16x16 block is two m16n8 tensor-core tiles, K = the
        // staged AO rows (up to 4 matched row blocks = 24 rows = 3 k-steps of 8).
        // Each product is split into TF32 hi + lo parts and summed as
        // hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), into
        // FP32 fragments flushed to FP64 every 32 of b's rows, as the FP64 path.
        float* bc = buf;                          // [kTcRows][kTcStride]: C[r, a] rows
        float* by = buf + kTcRows * kTcStride;    // [kTcRows][kTcStride]: Y[r, b] rows
        const int gq = lane >> 2, tq = lane & 3;
        for (int p = p0 + split + warp * n_split; p < p1; p += kTfWarps * n_split) {
            const int b = tp_b[p];
            const int nb = y_n[b];
            const int* yr = y_row + (size_t)b * capY;
            float acc[2][4];
            double accd[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[h][q] = 0.f;
                    accd[h][q] = 0.0;
                }
            for (int k0 = 0; k0 < nb; k0 += 32) {
                const int k = k0 + lane;
                const int rr = k < nb ? yr[k] : 0;
                const int sl = k < nb ? slot_of[rr - r0] : -1;
                unsigned m = __ballot_sync(0xffffffffu, sl >= 0);
                while (m) {
                    // up to kStage matched row blocks: their row, a's slot and b's position
                    int nst = 0, rowv[kStage], ssv[kStage], kkv[kStage];
#pragma unroll
                    for (int g = 0; g < kStage; ++g) {
                        const int src_lane = m ? __ffs(m) - 1 : 0;
                        if (m) {
                            m &= m - 1;
                            ++nst;
                        }
                        rowv[g] = __shfl_sync(0xffffffffu, rr, src_lane);
                        ssv[g] = __shfl_sync(0xffffffffu, sl, src_lane);
                        kkv[g] = k0 + src_lane;
                    }
                    // stage: lane q*4 + part (< 24) copies 16 bytes of AO row q of
                    // C[r, a] and of Y[r, b] for every staged row block, loads first
                    if (lane < 24) {
                        const int q = lane >> 2, part = lane & 3;
                        float4 cv[kStage], yv[kStage];
#pragma unroll
                        for (int g = 0; g < kStage; ++g)
                            if (g < nst) {
                                cv[g] = *((const float4*)(c_val + ((size_t)rowv[g] * cap + ssv[g]) * kTileVals +
                                                          q * 16) + part);
                                yv[g] = *((const float4*)(y_val + ((size_t)b * capY + kkv[g]) * kTileVals + q * 16) +
                                          part);
                            }
#pragma unroll
                        for (int g = 0; g < kStage; ++g)
                            if (g < nst) {
                                *(float4*)(bc + (g * kAoPerMol + q) * kTcStride + 4 * part) = cv[g];
                                *(float4*)(by + (g * kAoPerMol + q) * kTcStride + 4 * part) = yv[g];
                            }
                    }
                    __syncwarp();
                    const int nkr = nst * kAoPerMol;
                    for (int ks = 0; ks < nkr; ks += 8) {
                        const int ka = ks + tq, kb = ks + tq + 4;
                        const bool va = ka < nkr, vb = kb < nkr;
                        uint32_t ah[4], al[4];
                        split_tf32(va ? bc[ka * kTcStride + gq] : 0.f, ah[0], al[0]);
                        split_tf32(va ? bc[ka * kTcStride + gq + 8] : 0.f, ah[1], al[1]);
                        split_tf32(vb ? bc[kb * kTcStride + gq] : 0.f, ah[2], al[2]);
                        split_tf32(vb ? bc[kb * kTcStride + gq + 8] : 0.f, ah[3], al[3]);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            uint32_t bh[2], bl[2];
                            split_tf32(va ? by[ka * kTcStride + 8 * h + gq] : 0.f, bh[0], bl[0]);
                            split_tf32(vb ? by[kb * kTcStride + 8 * h + gq] : 0.f, bh[1], bl[1]);
                            mma_tf32(acc[h], al, bh);
                            mma_tf32(acc[h], ah, bl);
                            mma_tf32(acc[h], ah, bh);
                        }
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        accd[h][q] += (double)acc[h][q];
                        acc[h][q] = 0.f;
                    }
            }
            T* o = out + (size_t)tp_out[p] * 256;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                o[gq * 16 + 8 * h + 2 * tq] = (T)accd[h][0];
                o[gq * 16 + 8 * h + 2 * tq + 1] = (T)accd[h][1];
                o[(gq + 8) * 16 + 8 * h + 2 * tq] = (T)accd[h][2];
                o[(gq + 8) * 16 + 8 * h + 2 * tq + 1] = (T)accd[h][3];
            }
        }
        return;
    }
    const int i0 = 2 * (lane >> 2), j0 = 4 * (lane & 3);
    using A = typename Acc<T>::type;
    using VT = typename V4<T>::type;
    constexpr int kVec = sizeof(VT) / sizeof(T);          // values per 16-byte load
    constexpr int kPerTile = kTileVals / kVec;            // 16-byte loads per tile
    for (int p = p0 + split + warp * n_split; p < p1; p += kTfWarps * n_split) {
        const int b = tp_b[p];
        const int nb = y_n[b];
        const int* yr = y_row + (size_t)b * capY;
        double accd[8];
        A acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[q] = 0;
            accd[q] = 0.0;
        }
        for (int k0 = 0; k0 < nb; k0 += 32) {
            const int k = k0 + lane;
            const int s = k < nb ? slot_of[yr[k] - r0] : -1;
            unsigned m = __ballot_sync(0xffffffffu, s >= 0);
            while (m) {
                // stage up to kStage matched row blocks
                int rows[kStage];
                int nst = 0;
#pragma unroll
                for (int g = 0; g < kStage; ++g) {
                    rows[g] = -1;
                    if (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        rows[g] = src;
                        ++nst;
                    }
                }
#pragma unroll
                for (int g = 0; g < kStage; ++g) {
                    if (g >= nst) break;
                    const int ss = __shfl_sync(0xffffffffu, s, rows[g]);
                    const int kk = k0 + rows[g];
                    const int r = yr[kk];
                    const VT* cs = (const VT*)(c_val + ((size_t)r * cap + ss) * kTileVals);
                    const VT* ys = (const VT*)(y_val + ((size_t)b * capY + kk) * kTileVals);
                    VT* bc = (VT*)(buf + (size_t)g * 2 * kTileVals);
                    VT* by = (VT*)(buf + (size_t)g * 2 * kTileVals + kTileVals);
                    for (int v = lane; v < kPerTile; v += 32) {
                        bc[v] = cs[v];
                        by[v] = ys[v];
                    }
                }
                __syncwarp();
                for (int g = 0; g < nst; ++g) {
                    const T* bc = buf + (size_t)g * 2 * kTileVals;
                    const T* by = bc + kTileVals;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const A c0 = (A)bc[q * 16 + i0], c1 = (A)bc[q * 16 + i0 + 1];
                        const A y0 = (A)by[q * 16 + j0], y1 = (A)by[q * 16 + j0 + 1];
                        const A y2 = (A)by[q * 16 + j0 + 2], y3 = (A)by[q * 16 + j0 + 3];
                        acc[0] += c0 * y0;
                        acc[1] += c0 * y1;
                        acc[2] += c0 * y2;
                        acc[3] += c0 * y3;
                        acc[4] += c1 * y0;
                        acc[5] += c1 * y1;
                        acc[6] += c1 * y2;
                        acc[7] += c1 * y3;
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                accd[q] += (double)acc[q];
                acc[q] = 0;
            }
        }
        T* o = out + (size_t)tp_out[p] * 256;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            o[i0 * 16 + j0 + u] = (T)accd[u];
            o[(i0 + 1) * 16 + j0 + u] = (T)accd[4 + u];
        }
    }
}

// diag(F) per MO from the diagonal tile pairs
template <typename T>
__global__ void k_extract_diag(int n_tiles, const int* __restrict__ tile_mo0, const int* __restrict__ tile_nmo,
                               const T* __restrict__ Ft, double* __restrict__ Fd) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_tiles * 16) return;
    int t = idx >> 4, c = idx & 15;
    if (c < tile_nmo[t]) Fd[tile_mo0[t] + c] = (double)Ft[(size_t)t * 256 + c * 17];
}

// ---------------------------------------------------------------------------
// Density: P_mn = 2 sum_{occ tiles t in rows m and n} C[m,t] C[n,t]^T on the
// molecule-pair pattern; q_a += sum_{mu in a} sum_nu P_mu,nu S_mu,nu and the
// band energy sum P*H0 per molecule (Eq. pop). One CTA per row block m, one
// warp per neighbour n >= m (P_nm = P_mn^T): each pair's shares of q and of
// the band energy are written for both rows, and k_density_sum adds them per
// molecule in neighbour order.
// ---------------------------------------------------------------------------
constexpr int kDensWarps = 8;
constexpr int kDensFlush = 32;  // tiles per lane between FP64 flushes (FP32 sums of at most 32 products)
constexpr int kDensUnroll = 1;  // shared tiles per half-warp and round (2 measured no faster)
constexpr int kDensMinBlocks = 2;   // resident CTAs per SM the register budget aims at
template <typename T>
__global__ void __launch_bounds__(kDensWarps * 32, kDensMinBlocks)
k_density(int n_occ_tiles, int map_n, const int* __restrict__ mol_ot0, int cap, const int* __restrict__ c_nt,
          const int* __restrict__ c_tile, const T* __restrict__ c_val, const int* __restrict__ mp_ptr,
          const int* __restrict__ mp_col, const double* __restrict__ H0b, const double* __restrict__ Sb,
          const int* __restrict__ mp_rev, double2* __restrict__ dpart, double* __restrict__ P_out) {
    // slot of every occupied tile of m's cluster in row m, or -1 (map_n = largest cluster);
    // then, in mixed precision, the FP64 sums of each lane's 36 products (flushed
    // from FP32 every kDensFlush tiles), kept in shared memory to save registers
    extern __shared__ int smap[];
    constexpr bool kSplit = !std::is_same<typename Acc<T>::type, double>::value;
    double* sacc = (double*)(smap + ((map_n + 1) & ~1));   // [warp][36][32]: per-lane FP64 sums
    const int m = blockIdx.x;
    const int t0 = mol_ot0[m];
    // P_nm = P_mn^T: this CTA takes the pairs with n >= m (neighbour lists are
    // sorted) and hands each pair's share of the charges and of the band
    // energy to both rows
    __shared__ int s_jlo;
    if (threadIdx.x == 0) s_jlo = 0;
    for (int i = threadIdx.x; i < map_n; i += blockDim.x) smap[i] = -1;
    __syncthreads();
    for (int w = threadIdx.x; w < mp_ptr[m + 1] - mp_ptr[m]; w += blockDim.x)
        if (mp_col[mp_ptr[m] + w] < m) atomicAdd(&s_jlo, 1);
    const int ntm = c_nt[m];
    for (int s = threadIdx.x; s < ntm; s += blockDim.x) {
        int t = c_tile[(size_t)m * cap + s];
        if (t < n_occ_tiles) smap[t - t0] = s;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e0 = mp_ptr[m], ne = mp_ptr[m + 1] - e0;
    using A = typename Acc<T>::type;
    const int col = lane & 15, half = lane >> 4;
    for (int w = s_jlo + warp; w < ne; w += kDensWarps) {
        const int e = e0 + w;
        const int n = mp_col[e];
        A acc[36];
        double* wacc = sacc + (size_t)warp * 36 * 32 + lane;
        bool flushed = false;   // the first flush stores instead of adding
#pragma unroll
        for (int u = 0; u < 36; ++u) acc[u] = 0;
        const int ntn = c_nt[n];
        int since = 0;
        // 32 of n's tiles at a time: one coalesced load of their ids, the shared
        // ones found with one ballot; then each half-warp takes kDensUnroll shared
        // tiles per round, so their loads are in flight together
        for (int base = 0; base < ntn; base += 32) {
            const int s = base + lane;
            const int t = s < ntn ? c_tile[(size_t)n * cap + s] : n_occ_tiles;
            const int sm_ = t < n_occ_tiles ? smap[t - t0] : -1;
            unsigned mm = __ballot_sync(0xffffffffu, sm_ >= 0);
            const bool virt_seen = __any_sync(0xffffffffu, s < ntn && t >= n_occ_tiles);
            while (mm) {
                int src[kDensUnroll];
#pragma unroll
                for (int u = 0; u < kDensUnroll; ++u) {
                    // bits in order: half 0 takes the 1st, 3rd, ..., half 1 the 2nd, 4th, ...
                    int b0 = -1, b1 = -1;
                    if (mm) {
                        b0 = __ffs(mm) - 1;
                        mm &= mm - 1;
                    }
                    if (mm) {
                        b1 = __ffs(mm) - 1;
                        mm &= mm - 1;
                    }
                    src[u] = half ? b1 : b0;
                }
                A a6[kDensUnroll][6], b6[kDensUnroll][6];
#pragma unroll
                for (int u = 0; u < kDensUnroll; ++u) {
                    const int ss = __shfl_sync(0xffffffffu, s, src[u] < 0 ? 0 : src[u]);
                    const int sm2 = __shfl_sync(0xffffffffu, sm_, src[u] < 0 ? 0 : src[u]);
                    if (src[u] >= 0) {
                        const T* cm = c_val + ((size_t)m * cap + sm2) * kTileVals + col;
                        const T* cn = c_val + ((size_t)n * cap + ss) * kTileVals + col;
#pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            a6[u][k] = (A)cm[k * kTileW];
                            b6[u][k] = (A)cn[k * kTileW];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kDensUnroll; ++u) {
                    if (src[u] < 0) continue;
#pragma unroll
                    for (int k = 0; k < 6; ++k)
#pragma unroll
                        for (int l = 0; l < 6; ++l) acc[k * 6 + l] += a6[u][k] * b6[u][l];
                    if constexpr (kSplit) {
                        if (++since == kDensFlush) {
                            since = 0;
#pragma unroll
                            for (int v = 0; v < 36; ++v) {
                                wacc[v * 32] = flushed ? wacc[v * 32] + (double)acc[v] : (double)acc[v];
                                acc[v] = 0;
                            }
                            flushed = true;
                        }
                    }
                }
            }
            if (virt_seen) break;   // tiles are sorted: occupied tiles first
        }
        // lane sums to shared memory, then lane u < 36 adds up entry u over the
        // 32 lanes (rotated start: no bank conflicts) and weights it by S and H0
#pragma unroll
        for (int u = 0; u < 36; ++u) wacc[u * 32] = flushed ? wacc[u * 32] + (double)acc[u] : (double)acc[u];
        __syncwarp();
        // row sums of P o S by the atoms of m, column sums by the atoms of n
        // (AOs: O s, p, p, p, then H1 s, H2 s), and sum P o H0
        const bool self = n == m;
        const int er = self ? e : mp_rev[e];
        double qr[3] = {0, 0, 0}, qc[3] = {0, 0, 0}, eb = 0.0;
        for (int u = lane; u < 36; u += 32) {
            const double* row = sacc + ((size_t)warp * 36 + u) * 32;
            double v = 0.0;
            for (int j = 0; j < 32; ++j) v += row[(j + lane) & 31];
            const double P = 2.0 * v;
            const int k = u / 6, l = u - 6 * k;   // AO of m, AO of n
            if (P_out) {
                P_out[(size_t)e * 36 + u] = P;
                if (!self) P_out[(size_t)er * 36 + l * 6 + k] = P;
            }
            const double pq = P * Sb[(size_t)e * 36 + u];
            qr[0] += k < 4 ? pq : 0.0;
            qr[1] += k == 4 ? pq : 0.0;
            qr[2] += k == 5 ? pq : 0.0;
            qc[0] += l < 4 ? pq : 0.0;
            qc[1] += l == 4 ? pq : 0.0;
            qc[2] += l == 5 ? pq : 0.0;
            eb += P * H0b[(size_t)e * 36 + u];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                qr[i] += __shfl_xor_sync(0xffffffffu, qr[i], off);
                qc[i] += __shfl_xor_sync(0xffffffffu, qc[i], off);
            }
            eb += __shfl_xor_sync(0xffffffffu, eb, off);
        }
        __syncwarp();
        if (lane == 0) {
            dpart[2 * (size_t)e] = make_double2(qr[0], qr[1]);
            dpart[2 * (size_t)e + 1] = make_double2(qr[2], eb);
            if (!self) {
                dpart[2 * (size_t)er] = make_double2(qc[0], qc[1]);
                dpart[2 * (size_t)er + 1] = make_double2(qc[2], eb);
            }
        }
    }
}

// q and the band energy of every molecule: its pairs' shares summed in
// neighbour order
__global__ void k_density_sum(int n_mol, const int* __restrict__ mp_ptr, const double2* __restrict__ dpart,
                              double* __restrict__ q, double* __restrict__ e_mol) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mol) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int e = mp_ptr[m]; e < mp_ptr[m + 1]; ++e) {
        const double2 a = dpart[2 * (size_t)e], b = dpart[2 * (size_t)e + 1];
        s0 += a.x;
        s1 += a.y;
        s2 += b.x;
        s3 += b.y;
    }
    q[3 * m] = s0;
    q[3 * m + 1] = s1;
    q[3 * m + 2] = s2;
    e_mol[m] = s3;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static cudaError_t ensure_attrs();

cudaError_t launch_colindex(Ctx* c) {
    c->n_launch += 4;
    cudaError_t ea = ensure_attrs();
    if (ea != cudaSuccess) return ea;
    const int b = c->cur;
    cudaMemsetAsync(c->d_cci_cnt, 0, (size_t)c->n_tiles * 4, c->stream);
    k_ci_count<<<c->n_mol, 128, 0, c->stream>>>(c->n_mol, c->cap, c->d_c_nt[b], c->d_c_tile[b], c->d_cci_cnt);
    k_scan<<<1, 1024, 0, c->stream>>>(c->n_tiles, c->d_cci_cnt, c->d_cci_ptr);
    cudaMemsetAsync(c->d_cci_cnt, 0, (size_t)c->n_tiles * 4, c->stream);
    k_ci_fill<<<c->n_mol, 128, 0, c->stream>>>(c->n_mol, c->cap, c->d_c_nt[b], c->d_c_tile[b], c->d_cci_ptr,
                                               c->d_cci_cnt, c->d_cci_row, c->d_cci_slot);
    const size_t ssmem = (size_t)2 * ((c->max_cl_mol + 31) / 32) * 4;
    k_ci_sort<<<c->n_tiles, kSortThreads, ssmem, c->stream>>>(c->d_cci_ptr, c->d_cci_row, c->d_cci_slot,
                                                              c->d_tile_row0, c->max_cl_mol, &c->d_sc->err);
    return cudaGetLastError();
}

static bool g_attr_done[64] = {false};   // per device: function attributes are set per device

template <typename T>
static cudaError_t set_attrs() {
    cudaError_t e;
    e = cudaFuncSetAttribute(k_xc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_transform<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_transform<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_density<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return e;
}

static cudaError_t ensure_attrs() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && g_attr_done[dev]) return cudaSuccess;
    e = set_attrs<double>();
    if (e != cudaSuccess) return e;
    e = set_attrs<float>();
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_attr_done[dev] = true;
    return e;
}

cudaError_t launch_xc(Ctx* c, bool use_h, int tile_lo, int tile_hi, int own_below) {
    c->n_launch += 1;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    const int b = c->cur;
    const int n = tile_hi - tile_lo;
    if (n <= 0) return cudaSuccess;
    const int nr = c->max_cl_mol;
    const size_t smem = (size_t)((nr + 31) / 32) * 8 + (size_t)nr * 2 + 64;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (c->prec == SSCF_FP64)
        k_xc<double><<<n, 256, smem, c->stream>>>(tile_lo, nr, own_below, c->cap, c->capY, c->d_tile_row0, c->d_cci_ptr, c->d_cci_row,
                                                  c->d_cci_slot, (const double*)c->d_c_val[b], c->d_mp_ptr,
                                                  c->d_mp_col, (const double*)(use_h ? c->d_Hb : c->d_Sbt),
                                                  c->d_y_n, c->d_y_row, (double*)c->d_y_val, &c->d_sc->err);
    else
        k_xc<float><<<n, 256, smem, c->stream>>>(tile_lo, nr, own_below, c->cap, c->capY, c->d_tile_row0, c->d_cci_ptr, c->d_cci_row,
                                                 c->d_cci_slot, (const float*)c->d_c_val[b], c->d_mp_ptr,
                                                 c->d_mp_col, (const float*)(use_h ? c->d_Hb : c->d_Sbt),
                                                 c->d_y_n, c->d_y_row, (float*)c->d_y_val, &c->d_sc->err);
    return cudaGetLastError();
}

cudaError_t launch_xc_rot(Ctx* c) {
    // the occupied tiles enter the rotation transform only through their
    // diagonal tile pairs C[:, a]^T H C[:, a], whose sum runs over a's rows
    // (one launch for all tiles keeps the CTAs of both kinds in one grid)
    return launch_xc(c, true, 0, c->n_tiles, c->n_occ_tiles);
}

template <typename T>
static cudaError_t transform_t(Ctx* c, const int* ptr, const int* bl, const int* outl, void* out) {
    const size_t smem = (size_t)kTfWarps * tf_stage_vals<T>() * sizeof(T) + (size_t)c->max_cl_mol * 2;
    auto kern = c->tf_regs == 1 ? k_transform<T, 4> : k_transform<T, 1>;
    kern<<<c->n_tiles * c->tf_split, kTfWarps * 32, smem, c->stream>>>(
        c->tf_split, c->max_cl_mol, c->d_tile_row0, c->cap, c->capY, ptr, bl, outl, c->d_cci_ptr, c->d_cci_row,
        c->d_cci_slot, (const T*)c->d_c_val[c->cur], c->d_y_n, c->d_y_row, (const T*)c->d_y_val, (T*)out);
    return cudaGetLastError();
}

cudaError_t launch_transform_rot(Ctx* c) {
    c->n_launch += 3;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    if ((size_t)kTfWarps * (c->prec == SSCF_FP64 ? tf_stage_vals<double>() * 8 : tf_stage_vals<float>() * 4) +
            (size_t)c->max_cl_mol * 2 > 200 * 1024)
        return cudaErrorInvalidValue;
    if (c->prec == SSCF_FP64) {
        e = transform_t<double>(c, c->d_rot_tp_ptr, c->d_rot_tp_b, c->d_rot_tp_out, c->d_F);
        if (e == cudaSuccess)
            e = transform_t<double>(c, c->d_diag_tp_ptr, c->d_diag_tp_b, c->d_diag_tp_out, c->d_Fdiag_tiles);
        if (e == cudaSuccess)
            k_extract_diag<double><<<(c->n_tiles * 16 + 255) / 256, 256, 0, c->stream>>>(
                c->n_tiles, c->d_tile_mo0, c->d_tile_nmo, (const double*)c->d_Fdiag_tiles, c->d_Fd);
    } else {
        e = transform_t<float>(c, c->d_rot_tp_ptr, c->d_rot_tp_b, c->d_rot_tp_out, c->d_F);
        if (e == cudaSuccess)
            e = transform_t<float>(c, c->d_diag_tp_ptr, c->d_diag_tp_b, c->d_diag_tp_out, c->d_Fdiag_tiles);
        if (e == cudaSuccess)
            k_extract_diag<float><<<(c->n_tiles * 16 + 255) / 256, 256, 0, c->stream>>>(
                c->n_tiles, c->d_tile_mo0, c->d_tile_nmo, (const float*)c->d_Fdiag_tiles, c->d_Fd);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_transform_ortho(Ctx* c, int w) {
    c->n_launch += 1;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    if (c->prec == SSCF_FP64)
        return transform_t<double>(c, c->d_ort_tp_ptr[w], c->d_ort_tp_b[w], c->d_ort_tp_out[w], c->d_sig);
    return transform_t<float>(c, c->d_ort_tp_ptr[w], c->d_ort_tp_b[w], c->d_ort_tp_out[w], c->d_sig);
}

cudaError_t launch_density(Ctx* c, double* P_out) {
    c->n_launch += 2;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)((c->max_cl_otiles + 1) & ~1) * 4 + (size_t)kDensWarps * 36 * 32 * 8;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int b = c->cur;
    double2* dpart = (double2*)c->d_dens_part;
    if (c->prec == SSCF_FP64)
        k_density<double><<<c->n_mol, kDensWarps * 32, smem, c->stream>>>(
            c->n_occ_tiles, c->max_cl_otiles, c->d_mol_ot0, c->cap, c->d_c_nt[b], c->d_c_tile[b],
            (const double*)c->d_c_val[b], c->d_mp_ptr, c->d_mp_col, c->d_H0b, c->d_Sb, c->d_mp_rev, dpart, P_out);
    else
        k_density<float><<<c->n_mol, kDensWarps * 32, smem, c->stream>>>(
            c->n_occ_tiles, c->max_cl_otiles, c->d_mol_ot0, c->cap, c->d_c_nt[b], c->d_c_tile[b],
            (const float*)c->d_c_val[b], c->d_mp_ptr, c->d_mp_col, c->d_H0b, c->d_Sb, c->d_mp_rev, dpart, P_out);
    k_density_sum<<<(c->n_mol + 127) / 128, 128, 0, c->stream>>>(c->n_mol, c->d_mp_ptr, dpart, c->d_q, c->d_e_mol);
    return cudaGetLastError();
}

}  // namespace sscf
