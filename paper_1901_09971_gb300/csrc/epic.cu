// EPIC interpolation of the sparse flow into a dense field (Section 2,
// "Interpolation": an affine model fitted to the k nearest sparse vectors under a
// geodesic distance that penalises crossing image edges, the edges taken from
// image gradients; Section 3 "Parameters": k = 128). The paper gives no formulas;
// the reading, with every distance an exact integer, is stated with
// epic_interpolate in degraf.h.
//
// Launches on the caller's stream:
//   1. edge cost C = base + gain (|Gx| + |Gy|) per pixel (integer Sobel), labels cleared;
//   2. seeds claim their pixels (atomicMin on (distance 0, index)), then keep a
//      pixel only where they hold it;
//   3. geodesic Voronoi labelling by tile-local relaxation: 32 x 32 tiles iterate
//      min-plus updates of the packed key (distance << 24 | seed) in shared memory
//      until they are locally stable, write improvements back with atomicMin and
//      count them; passes repeat until one changes nothing (the host reads the
//      counter every four passes). Relaxation converges to the unique fixed
//      point, the lexicographic (distance, seed) minimum, whatever the order;
//   4-6. seed graph: links of 4-adjacent pixels in different cells are counted,
//      scanned into offsets and filled into per-seed lists (duplicates kept: the
//      search below takes their minimum);
//   7-8. each list keeps one link per neighbour (its smallest weight), and every
//      link records where its neighbour's list lies, so a search reads a popped
//      seed's links without first loading its list bounds;
//   9. per seed, one warp runs Dijkstra over the seed graph on (distance, index)
//      keys until k seeds are settled, with the frontier (128 entries), a hash of
//      discovered seeds and the settled list in shared memory (32 warps per SM);
//      then the warp fits the weighted affine model in FP64. A search whose
//      frontier outgrows 128 entries is queued and redone by a retry kernel with
//      room for 4096;
//   10. dense flow: every pixel evaluates its seed's model.
#include <math.h>

#include "common.cuh"

namespace {

constexpr unsigned long long kNone = ~0ull;
constexpr int kIdxBits = 24;
constexpr unsigned long long kIdxMask = (1ull << kIdxBits) - 1;
constexpr long long kDistLimit = 1ll << 40;  // the distance field of a packed key
constexpr int kTile = 32;                    // Voronoi tiles: 32 x 32 pixels, 32 x 8 threads
constexpr int kMaxPasses = 4096;
constexpr int kPassBatch = 4;
constexpr int kThreads = 256;

// Device status bits (any of them makes the call return DGF_ERR_DEVICE).
enum : int { kErrFrontier = 1, kErrHash = 2, kErrFill = 4, kErrRange = 8 };

__device__ __forceinline__ bool is_tracked(uint8_t s) { return s == DGF_TRACKED || s == DGF_MAXITER; }

__global__ void __launch_bounds__(kThreads) epic_cost_kernel(const uint8_t* img, int W, int H, int pitch, int base,
                                                             int gain, int* cost, unsigned long long* key)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    const int xm = max(x - 1, 0), xp = min(x + 1, W - 1);
    const uint8_t* r0 = img + (size_t)max(y - 1, 0) * pitch;
    const uint8_t* r1 = img + (size_t)y * pitch;
    const uint8_t* r2 = img + (size_t)min(y + 1, H - 1) * pitch;
    const int a = r0[xm], b = r0[x], c = r0[xp], d = r1[xm], f = r1[xp], g = r2[xm], h = r2[x], i = r2[xp];
    const int gx = (c - a) + 2 * (f - d) + (i - g);
    const int gy = (g - a) + 2 * (h - b) + (i - c);
    const size_t o = (size_t)y * W + x;
    cost[o] = base + gain * (abs(gx) + abs(gy));
    key[o] = kNone;
}

__global__ void __launch_bounds__(kThreads) epic_seed_kernel(const float2* pts, const uint8_t* status, int n, int W,
                                                             int H, unsigned long long* key, int* seed_pix)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    int o = -1;
    if (is_tracked(status[i])) {
        const float2 p = pts[i];
        // x + 1/2 is exact in FP32 below 2^22; NaN clamps to 0
        const int x = (int)fminf(fmaxf(floorf(p.x + 0.5f), 0.f), (float)(W - 1));
        const int y = (int)fminf(fmaxf(floorf(p.y + 0.5f), 0.f), (float)(H - 1));
        o = y * W + x;
        atomicMin(&key[o], (unsigned long long)i);  // distance 0: the lowest index holds the pixel
    }
    seed_pix[i] = o;
}

__global__ void __launch_bounds__(kThreads) epic_seed_owner_kernel(const unsigned long long* key, int n, int* seed_pix)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const int o = seed_pix[i];
    if (o >= 0 && key[o] != (unsigned long long)i) seed_pix[i] = -1;
}

__device__ __forceinline__ void relax(unsigned long long& best, unsigned long long kn, int w)
{
    if (kn != kNone) best = min(best, kn + ((unsigned long long)w << kIdxBits));
}

__global__ void __launch_bounds__(kThreads) epic_voronoi_kernel(const int* cost, unsigned long long* key, int W, int H,
                                                                int* changed, int pass)
{
    __shared__ unsigned long long sk[kTile + 2][kTile + 2];
    __shared__ int sc[kTile + 2][kTile + 2];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int e = tid; e < (kTile + 2) * (kTile + 2); e += kThreads) {
        const int ly = e / (kTile + 2), lx = e - ly * (kTile + 2);
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        unsigned long long k = kNone;
        int c = 0;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t o = (size_t)gy * W + gx;
            // halo keys belong to other tiles, which may lower them concurrently;
            // any value read is a valid upper bound
            k = *reinterpret_cast<const volatile unsigned long long*>(key + o);
            c = cost[o];
        }
        sk[ly][lx] = k;
        sc[ly][lx] = c;
    }
    __syncthreads();
    const int lx = threadIdx.x + 1;
    const bool xin = x0 + threadIdx.x < W;
    unsigned long long orig[kTile / 8];
#pragma unroll
    for (int r = 0; r < kTile / 8; ++r) orig[r] = sk[threadIdx.y + 8 * r + 1][lx];
    // Jacobi sweeps with the halo fixed; a sweep extends every shortest path by one
    // step, so the tile is stable after at most kTile^2 sweeps
    for (int it = 0; it <= kTile * kTile; ++it) {
        unsigned long long nk[kTile / 8];
        bool ch = false;
#pragma unroll
        for (int r = 0; r < kTile / 8; ++r) {
            const int ly = threadIdx.y + 8 * r + 1;
            unsigned long long best = sk[ly][lx];
            if (xin && y0 + ly - 1 < H) {
                const int c = sc[ly][lx];
                relax(best, sk[ly][lx - 1], sc[ly][lx - 1] + c);
                relax(best, sk[ly][lx + 1], sc[ly][lx + 1] + c);
                relax(best, sk[ly - 1][lx], sc[ly - 1][lx] + c);
                relax(best, sk[ly + 1][lx], sc[ly + 1][lx] + c);
                ch |= best < sk[ly][lx];
            }
            nk[r] = best;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kTile / 8; ++r) sk[threadIdx.y + 8 * r + 1][lx] = nk[r];
        if (!__syncthreads_or(ch)) break;
    }
    bool improved = false;
#pragma unroll
    for (int r = 0; r < kTile / 8; ++r) {
        const int ly = threadIdx.y + 8 * r + 1;
        const unsigned long long k = sk[ly][lx];
        if (k < orig[r]) {
            atomicMin(&key[(size_t)(y0 + ly - 1) * W + x0 + lx - 1], k);
            improved = true;
        }
    }
    if (__syncthreads_or(improved) && tid == 0) atomicAdd(&changed[pass], 1);
}

// Seed-graph links of pixel o with its right and lower neighbours.
template <bool FILL>
__global__ void __launch_bounds__(kThreads) epic_links_kernel(const unsigned long long* key, const int* cost, int W,
                                                              int H, int* cnt, const int* off, int* cur, int* adj_t,
                                                              long long* adj_w, int* err)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t o = (size_t)y * W + x;
    const unsigned long long k = key[o];
    if (k == kNone) return;
    const int s = (int)(k & kIdxMask);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q == 0 ? x + 1 >= W : y + 1 >= H) continue;
        const size_t o2 = q == 0 ? o + 1 : o + W;
        const unsigned long long k2 = key[o2];
        if (k2 == kNone || (int)(k2 & kIdxMask) == s) continue;
        const int t = (int)(k2 & kIdxMask);
        if (!FILL) {
            atomicAdd(&cnt[s], 1);
            atomicAdd(&cnt[t], 1);
            continue;
        }
        const long long w = (long long)(k >> kIdxBits) + cost[o] + cost[o2] + (long long)(k2 >> kIdxBits);
        const int ps = atomicAdd(&cur[s], 1), pt = atomicAdd(&cur[t], 1);
        if (ps < off[s + 1]) {
            adj_t[ps] = t;
            adj_w[ps] = w;
        } else {
            atomicOr(err, kErrFill);
        }
        if (pt < off[t + 1]) {
            adj_t[pt] = s;
            adj_w[pt] = w;
        } else {
            atomicOr(err, kErrFill);
        }
    }
}

// Exclusive scan of the link counts into offsets (off[n] = total) and cursors: one
// block walks the counts in coalesced tiles of 1024, carrying the running total.
__global__ void __launch_bounds__(1024) epic_scan_kernel(const int* cnt, int n, int* off, int* cur)
{
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + t;
        const int v = i < n ? cnt[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int z = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            wsum[lane] = z;
        }
        __syncthreads();
        const int excl = carry + (w ? wsum[w - 1] : 0) + x - v;
        if (i < n) {
            off[i] = excl;
            cur[i] = excl;
        }
        carry += wsum[31];
        __syncthreads();
    }
    if (t == 0) off[n] = carry;
}

// Per seed: keeps one link per neighbour (the smallest weight), compacting the list
// in place; end[s] becomes the end of the compacted list. One warp per seed walks
// the list in chunks of 32: lanes holding the same neighbour find each other with
// match.any and take their minimum weight; the lowest of them either lowers the
// weight of a link kept from an earlier chunk or appends a new one. The kept prefix
// never reaches the unread part of the list.
__global__ void __launch_bounds__(kThreads) epic_dedupe_kernel(const int* off, int* end, int* adj_t, long long* adj_w,
                                                               int n)
{
    const int lane = threadIdx.x & 31;
    const int s = (int)(((size_t)blockIdx.x * kThreads + threadIdx.x) >> 5);
    if (s >= n) return;  // warp-uniform
    const int b = off[s], e = off[s + 1];
    int out = b;
    for (int c = b; c < e; c += 32) {
        const bool has = c + lane < e;
        const int t = has ? adj_t[c + lane] : -1 - lane;  // empty lanes match nobody
        const long long w = has ? adj_w[c + lane] : 0;
        const unsigned grp = __match_any_sync(0xffffffffu, t);
        long long mw = w;
        for (int j = 0; j < 32; ++j) {
            const long long wj = __shfl_sync(0xffffffffu, w, j);
            if ((grp >> j) & 1u) mw = min(mw, wj);
        }
        const bool leader = has && lane == __ffs(grp) - 1;
        int found = -1;
        if (leader)
            for (int j = b; j < out; ++j)
                if (adj_t[j] == t) {
                    found = j;
                    break;
                }
        if (found >= 0 && mw < adj_w[found]) adj_w[found] = mw;  // leaders hold distinct neighbours
        const bool app = leader && found < 0;
        const unsigned km = __ballot_sync(0xffffffffu, app);
        __syncwarp();
        if (app) {
            const int pos = out + __popc(km & ((1u << lane) - 1));
            adj_t[pos] = t;
            adj_w[pos] = mw;
        }
        out += __popc(km);
        __syncwarp();
    }
    if (lane == 0) end[s] = out;
}

// Link records for the search: (neighbour, its list begin, its list end).
__global__ void __launch_bounds__(kThreads) epic_link_meta_kernel(const int* off, const int* end, const int* adj_t,
                                                                  int4* adj_i, int n)
{
    const int s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= n) return;
    for (int i = off[s], e = end[s]; i < e; ++i) {
        const int t = adj_t[i];
        adj_i[i] = make_int4(t, off[t], end[t], 0);
    }
}

struct KnnArgs {
    const float2* pts;
    const float2* flow;
    const int* seed_pix;
    const int* off;
    const int* end;
    const int4* adj_i;
    const long long* adj_w;
    double* models;  // [n][6]
    int* err;
    int* retry_count;
    int* retry_list;
    int32_t* knn_idx;
    int64_t* knn_dist;
    int32_t* knn_count;
    double* dbg_models;
    uint8_t* fit_kind;
    int n, k, model, cost_base;
    double a, min_spread2;
};

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// Per-warp shared layout of one search with a frontier of FCAP entries and a hash
// of HCAP slots: frontier keys (distance << 24 | index), their link-list bounds and
// hash slots; hash keys and values (frontier slot of a discovered seed, -2 once
// settled); then the settled list (index, distance).
template <int FCAP, int HCAP>
struct KnnLayout {
    static_assert((HCAP & (HCAP - 1)) == 0 && HCAP <= 32768 && FCAP <= 32767, "hash and frontier sizes");
    static constexpr int hash_bits = ilog2(HCAP);
    static constexpr size_t o_fmeta = (size_t)FCAP * 8;
    static constexpr size_t o_fhs = o_fmeta + (size_t)FCAP * 8;
    static constexpr size_t o_hkey = (o_fhs + (size_t)FCAP * 2 + 15) & ~(size_t)15;
    static constexpr size_t o_hval = o_hkey + (size_t)HCAP * 4;
    static constexpr size_t fixed = (o_hval + (size_t)HCAP * 2 + 15) & ~(size_t)15;
    __host__ __device__ static constexpr size_t o_sdist(int k) { return (fixed + (size_t)k * 4 + 7) & ~(size_t)7; }
    __host__ __device__ static constexpr size_t warp_bytes(int k) { return o_sdist(k) + (size_t)k * 8; }
};

// The fast search holds every frontier seen on the benchmark scenes (at most 73
// entries at k = 128); a search that outgrows it is redone by the retry kernel with
// room for 4096.
constexpr int kFastF = 128, kFastH = 512, kFastWarps = 8;
constexpr int kBigF = 4096, kBigH = 8192, kRetryBlocks = 152;
constexpr int kRetry = 16;  // search status: capacity exceeded, redo with the large layout

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dijkstra over the seed graph from seed s on (distance, index) keys until k seeds
// are settled; the warp's 32 lanes scan the frontier and relax one link each.
// Returns 0 with the settled list in shared memory, kRetry when the frontier or the
// hash is full, or kErrRange when a distance leaves the key's 40 bits.
template <int FCAP, int HCAP>
__device__ int knn_search(const KnnArgs& a, int s, unsigned char* base, int& cnt_out)
{
    using Lay = KnnLayout<FCAP, HCAP>;
    unsigned long long* fkey = reinterpret_cast<unsigned long long*>(base);
    int2* fmeta = reinterpret_cast<int2*>(base + Lay::o_fmeta);
    short* fhs = reinterpret_cast<short*>(base + Lay::o_fhs);
    int* hkey = reinterpret_cast<int*>(base + Lay::o_hkey);
    volatile int* vh = hkey;
    short* hval = reinterpret_cast<short*>(base + Lay::o_hval);
    int* sidx = reinterpret_cast<int*>(base + Lay::fixed);
    long long* sdist = reinterpret_cast<long long*>(base + Lay::o_sdist(a.k));
    const int lane = threadIdx.x & 31;
    auto slot_of = [](int t) { return (int)(((unsigned)t * 0x9E3779B1u) >> (32 - Lay::hash_bits)); };

    for (int j = lane; j < HCAP; j += 32) hkey[j] = -1;
    __syncwarp();
    if (lane == 0) {
        const int h = slot_of(s);
        hkey[h] = s;
        hval[h] = 0;
        fkey[0] = (unsigned long long)s;  // distance 0
        fhs[0] = (short)h;
        fmeta[0] = make_int2(a.off[s], a.end[s]);
    }
    __syncwarp();
    int fsize = 1, cnt = 0, status = 0;
    while (cnt < a.k && fsize > 0) {
        // pop the smallest key: lane minima with their slots, then two 32-bit warp minima
        unsigned long long best = kNone;
        int bslot = -1;
        for (int j = lane; j < fsize; j += 32) {
            const unsigned long long v = fkey[j];
            if (v < best) {
                best = v;
                bslot = j;
            }
        }
        const unsigned mhi = __reduce_min_sync(0xffffffffu, (unsigned)(best >> 32));
        const unsigned mlo = __reduce_min_sync(0xffffffffu, (unsigned)(best >> 32) == mhi ? (unsigned)best : ~0u);
        const unsigned long long gmin = ((unsigned long long)mhi << 32) | mlo;
        const unsigned own = __ballot_sync(0xffffffffu, bslot >= 0 && best == gmin);
        if (own == 0) {  // every frontier entry holds a key, so this cannot happen
            status = kErrFrontier;
            break;
        }
        const int slot = __shfl_sync(0xffffffffu, bslot, __ffs(own) - 1);
        const int u = (int)(gmin & kIdxMask);
        const long long d = (long long)(gmin >> kIdxBits);
        const int2 m = fmeta[slot];
        const bool last = cnt + 1 == a.k;  // the k-th seed's links are not needed
        const int nlk = last ? 0 : m.y - m.x;
        int4 li = make_int4(-1, 0, 0, 0);
        long long lw = 0;
        if (lane < nlk) {  // issue the first links' loads before the bookkeeping
            li = a.adj_i[m.x + lane];
            lw = a.adj_w[m.x + lane];
        }
        __syncwarp();
        if (lane == 0) {
            hval[fhs[slot]] = -2;
            const int L = fsize - 1;
            if (slot != L) {
                fkey[slot] = fkey[L];
                fhs[slot] = fhs[L];
                fmeta[slot] = fmeta[L];
                hval[fhs[slot]] = (short)slot;
            }
            sidx[cnt] = u;
            sdist[cnt] = d;
        }
        --fsize;
        ++cnt;
        __syncwarp();
        for (int c0 = 0; c0 < nlk; c0 += 32) {
            if (c0 > 0) {
                li = make_int4(-1, 0, 0, 0);
                if (c0 + lane < nlk) {
                    li = a.adj_i[m.x + c0 + lane];
                    lw = a.adj_w[m.x + c0 + lane];
                }
            }
            const bool has = c0 + lane < nlk;
            const int t = li.x;
            const long long nd = d + lw;
            int hs = -1, st = 0;
            bool isnew = false;
            if (has) {
                if (nd >= kDistLimit) st |= kErrRange;
                int h = slot_of(t);
                for (int q = 0; q < HCAP; ++q) {
                    const int c = vh[h];
                    if (c == t) {
                        hs = h;
                        break;
                    }
                    if (c == -1) {
                        const int prev = atomicCAS(&hkey[h], -1, t);
                        if (prev == -1 || prev == t) {
                            hs = h;
                            isnew = prev == -1;
                            break;
                        }
                    }
                    h = (h + 1) & (HCAP - 1);
                }
                if (hs < 0) st |= kRetry;
            }
            __syncwarp();
            const unsigned nm = __ballot_sync(0xffffffffu, isnew);
            if (isnew) {
                const int fs = fsize + __popc(nm & ((1u << lane) - 1));
                if (fs < FCAP) {
                    fkey[fs] = kNone;
                    fhs[fs] = (short)hs;
                    fmeta[fs] = make_int2(li.y, li.z);
                    hval[hs] = (short)fs;
                } else {
                    st |= kRetry;
                }
            }
            fsize = min(fsize + __popc(nm), FCAP);
            __syncwarp();
            if (has && hs >= 0 && !st) {
                const int v = hval[hs];
                if (v >= 0) atomicMin(&fkey[v], ((unsigned long long)nd << kIdxBits) | (unsigned long long)t);
            }
            __syncwarp();
            status = __reduce_or_sync(0xffffffffu, st);
            if (status) break;
        }
        if (status) break;
    }
    cnt_out = cnt;
    return status & kErrRange ? kErrRange : status;
}

// The weighted affine fit of seed s over its settled list (FP64; the 3 x 3 normal
// equations lose too many digits in FP32 when a neighbourhood is narrow) and the
// outputs. M = sum w v v^T, v = (x_t - x_s, y_t - y_s, 1).
__device__ void knn_fit_write(const KnnArgs& a, int s, int cnt, const int* sidx, const long long* sdist)
{
    const int lane = threadIdx.x & 31, k = a.k;
    if (a.knn_count && lane == 0) a.knn_count[s] = cnt;
    if (a.knn_idx)
        for (int j = lane; j < cnt; j += 32) {
            a.knn_idx[(size_t)s * k + j] = sidx[j];
            a.knn_dist[(size_t)s * k + j] = sdist[j];
        }
    const float2 ps = a.pts[s];
    double m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0, u0 = 0, u1 = 0, u2 = 0, v0 = 0, v1 = 0, v2 = 0;
    for (int j = lane; j < cnt; j += 32) {
        const int t = sidx[j];
        const double w = exp(-a.a * (double)sdist[j] / (2.0 * a.cost_base));
        const float2 pt = a.pts[t], ft = a.flow[t];
        const double vx = (double)pt.x - (double)ps.x, vy = (double)pt.y - (double)ps.y;
        const double fu = ft.x, fv = ft.y;
        m00 += w * vx * vx; m01 += w * vx * vy; m02 += w * vx;
        m11 += w * vy * vy; m12 += w * vy; m22 += w;
        u0 += w * vx * fu; u1 += w * vy * fu; u2 += w * fu;
        v0 += w * vx * fv; v1 += w * vy * fv; v2 += w * fv;
    }
    m00 = warp_sum(m00); m01 = warp_sum(m01); m02 = warp_sum(m02);
    m11 = warp_sum(m11); m12 = warp_sum(m12); m22 = warp_sum(m22);
    u0 = warp_sum(u0); u1 = warp_sum(u1); u2 = warp_sum(u2);
    v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
    if (lane != 0) return;
    // affine only with 3+ neighbours whose weighted position covariance (the Schur
    // complement of the constant term over sum w) has lambda_min >= min_spread^2
    bool affine = a.model == 1 && cnt >= 3;
    if (affine) {
        const double mx = m02 / m22, my = m12 / m22;
        const double cxx = m00 / m22 - mx * mx, cxy = m01 / m22 - mx * my, cyy = m11 / m22 - my * my;
        const double h = 0.5 * (cxx - cyy);
        affine = 0.5 * (cxx + cyy) - sqrt(h * h + cxy * cxy) >= a.min_spread2;
    }
    double A00 = 0, A01 = 0, A10 = 0, A11 = 0, b0 = u2 / m22, b1 = v2 / m22;
    if (affine) {
        // Cholesky of M = L L^T, then forward and back substitution for both flow components
        const double l00 = sqrt(m00), l10 = m01 / l00, l20 = m02 / l00;
        const double l11 = sqrt(m11 - l10 * l10), l21 = (m12 - l20 * l10) / l11;
        const double l22 = sqrt(m22 - l20 * l20 - l21 * l21);
        const double zu0 = u0 / l00, zu1 = (u1 - l10 * zu0) / l11, zu2 = (u2 - l20 * zu0 - l21 * zu1) / l22;
        const double zv0 = v0 / l00, zv1 = (v1 - l10 * zv0) / l11, zv2 = (v2 - l20 * zv0 - l21 * zv1) / l22;
        b0 = zu2 / l22;
        A01 = (zu1 - l21 * b0) / l11;
        A00 = (zu0 - l10 * A01 - l20 * b0) / l00;
        b1 = zv2 / l22;
        A11 = (zv1 - l21 * b1) / l11;
        A10 = (zv0 - l10 * A11 - l20 * b1) / l00;
    }
    double* mo = a.models + 6 * (size_t)s;
    mo[0] = A00; mo[1] = A01; mo[2] = A10; mo[3] = A11; mo[4] = b0; mo[5] = b1;
    if (a.dbg_models) {
        double* dm = a.dbg_models + 6 * (size_t)s;
        dm[0] = A00; dm[1] = A01; dm[2] = A10; dm[3] = A11; dm[4] = b0; dm[5] = b1;
    }
    if (a.fit_kind) a.fit_kind[s] = affine ? 1 : 2;
}

// One warp per seed with the fast layout; searches that outgrow it are queued for
// the retry kernel.
__global__ void __launch_bounds__(kFastWarps * 32) epic_knn_fit_kernel(KnnArgs a)
{
    using Lay = KnnLayout<kFastF, kFastH>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s = blockIdx.x * kFastWarps + wid;
    if (s >= a.n) return;  // warp-uniform
    if (a.seed_pix[s] < 0) {
        if (lane == 0) {
            if (a.knn_count) a.knn_count[s] = 0;
            if (a.fit_kind) a.fit_kind[s] = 0;
        }
        if (lane < 6) {
            a.models[6 * (size_t)s + lane] = 0.0;
            if (a.dbg_models) a.dbg_models[6 * (size_t)s + lane] = 0.0;
        }
        return;
    }
    unsigned char* base = smem + (size_t)wid * Lay::warp_bytes(a.k);
    int cnt = 0;
    const int st = knn_search<kFastF, kFastH>(a, s, base, cnt);
    if (st == kRetry) {
        if (lane == 0) a.retry_list[atomicAdd(a.retry_count, 1)] = s;
        return;
    }
    if (st) {
        if (lane == 0) atomicOr(a.err, st);
        return;
    }
    knn_fit_write(a, s, cnt, reinterpret_cast<const int*>(base + Lay::fixed),
                  reinterpret_cast<const long long*>(base + Lay::o_sdist(a.k)));
}

// The queued searches with room for 4096 frontier entries, one warp per block.
__global__ void __launch_bounds__(32) epic_knn_retry_kernel(KnnArgs a)
{
    using Lay = KnnLayout<kBigF, kBigH>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int total = *a.retry_count;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const int s = a.retry_list[i];
        int cnt = 0;
        const int st = knn_search<kBigF, kBigH>(a, s, smem, cnt);
        if (st) {
            if ((threadIdx.x & 31) == 0) atomicOr(a.err, st == kRetry ? kErrFrontier : st);
            continue;
        }
        knn_fit_write(a, s, cnt, reinterpret_cast<const int*>(smem + Lay::fixed),
                      reinterpret_cast<const long long*>(smem + Lay::o_sdist(a.k)));
    }
}

__global__ void __launch_bounds__(kThreads) epic_dense_kernel(const unsigned long long* key, const double* models,
                                                              const float2* pts, int W, int H, float2* dense,
                                                              int32_t* labels, int64_t* dist)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t o = (size_t)y * W + x;
    const unsigned long long k = key[o];
    if (k == kNone) {
        dense[o] = make_float2(0.f, 0.f);
        if (labels) labels[o] = -1;
        if (dist) dist[o] = -1;
        return;
    }
    const int s = (int)(k & kIdxMask);
    const double* m = models + 6 * (size_t)s;
    const float2 p = pts[s];
    const double dx = (double)x - (double)p.x, dy = (double)y - (double)p.y;
    dense[o] = make_float2((float)(m[0] * dx + m[1] * dy + m[4]), (float)(m[2] * dx + m[3] * dy + m[5]));
    if (labels) labels[o] = s;
    if (dist) dist[o] = (int64_t)(k >> kIdxBits);
}

// Workspace layout (256-byte aligned sections).
struct EpicLayout {
    size_t key, cost, seed_pix, cnt, off, cur, adj_t, adj_w, adj_i, models, retry, counters, total;
};

EpicLayout epic_layout(int W, int H, int n)
{
    const size_t np = (size_t)W * H, nl = 4 * np;  // at most two links per pixel, stored both ways
    EpicLayout L;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t o = at;
        at = dgf::round_up(at + bytes, 256);
        return o;
    };
    L.key = take(np * 8);
    L.cost = take(np * 4);
    L.seed_pix = take((size_t)n * 4);
    L.cnt = take((size_t)n * 4);
    L.off = take(((size_t)n + 1) * 4);
    L.cur = take((size_t)n * 4);
    L.adj_t = take(nl * 4);
    L.adj_w = take(nl * 8);
    L.adj_i = take(nl * 16);
    L.models = take((size_t)n * 48);
    L.retry = take((size_t)n * 4);
    L.counters = take((kMaxPasses + 2) * 4);  // pass counters, the status word, the retry count
    L.total = at;
    return L;
}

bool params_ok(const dgf_epic_params* p)
{
    return p && p->version == DGF_EPIC_PARAMS_VERSION && p->k >= 1 && p->k <= DGF_EPIC_MAX_K &&
           (p->model == 0 || p->model == 1) && p->cost_base >= 1 && p->cost_base <= 4096 && p->cost_gain >= 0 &&
           p->cost_gain <= 32 && p->a >= 0.0 && p->a < 1e30 && p->min_spread >= 0.0 && p->min_spread < 1e30;
}

}  // namespace

extern "C" int dgf_epic_params_default(dgf_epic_params* p)
{
    if (!p) return DGF_ERR_ARG;
    p->version = DGF_EPIC_PARAMS_VERSION;
    p->k = 128;
    p->model = 1;
    p->cost_base = 4;
    p->cost_gain = 1;
    p->a = 0.1;
    p->min_spread = 1.0;
    return DGF_OK;
}

extern "C" size_t dgf_epic_workspace(int W, int H, int n)
{
    if (W < 1 || H < 1 || n < 0 || W + H > DGF_EPIC_MAX_W_PLUS_H || n > DGF_EPIC_MAX_POINTS) return 0;
    return epic_layout(W, H, n).total;
}

extern "C" int epic_interpolate(const uint8_t* img, int W, int H, int pitch, const float* pts, const float* flow,
                                const uint8_t* status, int n, const dgf_epic_params* p, float* dense,
                                const dgf_epic_debug* dbg, void* workspace, size_t ws_bytes, cudaStream_t stream)
{
    if (!params_ok(p) || W < 1 || H < 1 || W + H > DGF_EPIC_MAX_W_PLUS_H || pitch < W || n < 0 ||
        n > DGF_EPIC_MAX_POINTS || !img || !dense || !workspace || (n > 0 && (!pts || !flow || !status)))
        return DGF_ERR_ARG;
    if (!dgf::aligned(dense, 8) || !dgf::aligned(workspace, 256) || (n > 0 && (!dgf::aligned(pts, 8) || !dgf::aligned(flow, 8))))
        return DGF_ERR_ARG;
    dgf_epic_debug d = {};
    if (dbg) d = *dbg;
    if ((d.knn_idx == nullptr) != (d.knn_dist == nullptr)) return DGF_ERR_ARG;
    if ((d.labels && !dgf::aligned(d.labels, 4)) || (d.dist && !dgf::aligned(d.dist, 8)) || (d.knn_idx && !dgf::aligned(d.knn_idx, 4)) ||
        (d.knn_dist && !dgf::aligned(d.knn_dist, 8)) || (d.knn_count && !dgf::aligned(d.knn_count, 4)) ||
        (d.models && !dgf::aligned(d.models, 8)) || (d.retried && !dgf::aligned(d.retried, 4)))
        return DGF_ERR_ARG;
    const EpicLayout L = epic_layout(W, H, n);
    if (ws_bytes < L.total) return DGF_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    auto* key = reinterpret_cast<unsigned long long*>(ws + L.key);
    auto* cost = reinterpret_cast<int*>(ws + L.cost);
    auto* seed_pix = reinterpret_cast<int*>(ws + L.seed_pix);
    auto* cnt = reinterpret_cast<int*>(ws + L.cnt);
    auto* off = reinterpret_cast<int*>(ws + L.off);
    auto* cur = reinterpret_cast<int*>(ws + L.cur);
    auto* adj_t = reinterpret_cast<int*>(ws + L.adj_t);
    auto* adj_w = reinterpret_cast<long long*>(ws + L.adj_w);
    auto* adj_i = reinterpret_cast<int4*>(ws + L.adj_i);
    auto* retry_list = reinterpret_cast<int*>(ws + L.retry);
    auto* models = reinterpret_cast<double*>(ws + L.models);
    auto* changed = reinterpret_cast<int*>(ws + L.counters);
    int* err = changed + kMaxPasses;
    int* retry_count = err + 1;
    const float2* p2 = reinterpret_cast<const float2*>(pts);
    const float2* f2 = reinterpret_cast<const float2*>(flow);

    if (cudaMemsetAsync(changed, 0, (kMaxPasses + 2) * sizeof(int), stream) != cudaSuccess) return DGF_ERR_CUDA;
    if (n > 0 && cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), stream) != cudaSuccess) return DGF_ERR_CUDA;
    const dim3 pix_block(32, 8), pix_grid((W + 31) / 32, (H + 7) / 8);
    const unsigned pt_grid = (unsigned)((n + kThreads - 1) / kThreads);
    epic_cost_kernel<<<pix_grid, pix_block, 0, stream>>>(img, W, H, pitch, p->cost_base, p->cost_gain, cost, key);
    if (n > 0) {
        epic_seed_kernel<<<pt_grid, kThreads, 0, stream>>>(p2, status, n, W, H, key, seed_pix);
        epic_seed_owner_kernel<<<pt_grid, kThreads, 0, stream>>>(key, n, seed_pix);
    }
    int rc = dgf::launch_status();
    if (rc != DGF_OK) return rc;

    // geodesic Voronoi labelling: passes until one changes nothing
    const dim3 tile_grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
    int pass = 0;
    for (;;) {
        for (int b = 0; b < kPassBatch && pass < kMaxPasses; ++b, ++pass)
            epic_voronoi_kernel<<<tile_grid, pix_block, 0, stream>>>(cost, key, W, H, changed, pass);
        if ((rc = dgf::launch_status()) != DGF_OK) return rc;
        int last = 0;
        if (cudaMemcpyAsync(&last, changed + pass - 1, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return DGF_ERR_CUDA;
        if (last == 0) break;
        if (pass >= kMaxPasses) return DGF_ERR_TIMEOUT;
    }

    if (n > 0) {
        epic_links_kernel<false><<<pix_grid, pix_block, 0, stream>>>(key, cost, W, H, cnt, nullptr, nullptr, nullptr,
                                                                     nullptr, err);
        epic_scan_kernel<<<1, 1024, 0, stream>>>(cnt, n, off, cur);
        epic_links_kernel<true><<<pix_grid, pix_block, 0, stream>>>(key, cost, W, H, nullptr, off, cur, adj_t, adj_w,
                                                                    err);
        epic_dedupe_kernel<<<(unsigned)((n + kThreads / 32 - 1) / (kThreads / 32)), kThreads, 0, stream>>>(
            off, cur, adj_t, adj_w, n);
        epic_link_meta_kernel<<<pt_grid, kThreads, 0, stream>>>(off, cur, adj_t, adj_i, n);
        KnnArgs a;
        a.pts = p2;
        a.flow = f2;
        a.seed_pix = seed_pix;
        a.off = off;
        a.end = cur;
        a.adj_i = adj_i;
        a.adj_w = adj_w;
        a.models = models;
        a.err = err;
        a.retry_count = retry_count;
        a.retry_list = retry_list;
        a.knn_idx = d.knn_idx;
        a.knn_dist = d.knn_dist;
        a.knn_count = d.knn_count;
        a.dbg_models = d.models;
        a.fit_kind = d.fit_kind;
        a.n = n;
        a.k = p->k;
        a.model = p->model;
        a.cost_base = p->cost_base;
        a.a = p->a;
        a.min_spread2 = p->min_spread * p->min_spread;
        const size_t smem_fast = KnnLayout<kFastF, kFastH>::warp_bytes(p->k) * kFastWarps;
        const size_t smem_big = KnnLayout<kBigF, kBigH>::warp_bytes(p->k);
        if (cudaFuncSetAttribute(epic_knn_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fast) !=
                cudaSuccess ||
            cudaFuncSetAttribute(epic_knn_retry_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_big) !=
                cudaSuccess)
            return DGF_ERR_CUDA;
        epic_knn_fit_kernel<<<(unsigned)((n + kFastWarps - 1) / kFastWarps), kFastWarps * 32, smem_fast, stream>>>(a);
        epic_knn_retry_kernel<<<kRetryBlocks, 32, smem_big, stream>>>(a);
    }
    epic_dense_kernel<<<pix_grid, pix_block, 0, stream>>>(key, models, p2, W, H, reinterpret_cast<float2*>(dense),
                                                          d.labels, d.dist);
    if (d.retried &&
        cudaMemcpyAsync(d.retried, retry_count, sizeof(int), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return DGF_ERR_CUDA;
    if ((rc = dgf::launch_status()) != DGF_OK) return rc;
    int status_word = 0;
    if (cudaMemcpyAsync(&status_word, err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return DGF_ERR_CUDA;
    return status_word ? DGF_ERR_DEVICE : DGF_OK;
}
