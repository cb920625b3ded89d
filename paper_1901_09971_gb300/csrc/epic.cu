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
//      scanned into offsets (three launches: block scans, a scan of the block
//      totals, the block offsets added) and filled into per-seed lists;
//   7-8. each list keeps one link per neighbour (its smallest weight), and every
//      link records where its neighbour's list lies, so a search reads a popped
//      seed's links without first loading its list bounds;
//   9. per seed, one warp runs Dijkstra over the seed graph with batch settling
//      (every frontier seed within its smallest incoming link of the frontier
//      minimum is final, so about 14 steps settle the 128 nearest instead of 128
//      pops), a hash of discovered seeds in shared memory, then sorts the settled
//      (distance, index) keys and fits the weighted affine model to the first k
//      (double-float sums, FP64 solve). A search that outgrows the hash (384 seeds;
//      1024 for k > 160) or the sort buffer (256; 512) is queued and redone by a
//      retry kernel with room for 8192;
//   10. dense flow: every pixel evaluates its seed's model.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr unsigned long long kNone = ~0ull;
constexpr int kIdxBits = 24;
constexpr unsigned long long kIdxMask = (1ull << kIdxBits) - 1;
constexpr long long kDistLimit = 1ll << 40;  // the distance field of a packed key
constexpr int kTile = 32;                    // Voronoi tiles: 32 x 32 pixels, 32 x 8 threads
constexpr int kMaxPasses = 4096;
constexpr int kThreads = 256;

constexpr long long kNoLink = 0xffffffffll;  // min link weight of a seed without links

// Device status bits (any of them makes the call return DGF_ERR_DEVICE).
enum : int { kErrFrontier = 1, kErrFill = 4, kErrRange = 8, kErrPasses = 16, kErrSync = 32 };
constexpr unsigned kBarrierTries = 1u << 24;  // polls (100 ns naps) before a grid barrier gives up

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

// One relaxation pass over the 32 x 32 tile at (x0, y0): the tile and a one-pixel
// halo in shared memory, Jacobi min-plus sweeps until the tile is stable, improved
// keys written back with atomicMin; counts the tile in changed[pass] if any key
// improved. Called by every thread of the block.
__device__ __forceinline__ void voronoi_tile(const int* cost, unsigned long long* key, int W, int H, int* changed,
                                             int pass, int x0, int y0)
{
    __shared__ unsigned long long sk[kTile + 2][kTile + 2];
    __shared__ int sc[kTile + 2][kTile + 2];
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
    __syncthreads();  // the next tile reuses sk and sc
}

// Barrier of all blocks of a cooperative launch (all co-resident): arrivals on a
// counter that grows by the grid size per use; the waits are bounded, and false
// comes back once a block gave up.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();  // this block's key and counter updates before its arrival
        atomicAdd(count, 1u);
        int ok = 0;
        for (unsigned i = 0; i < kBarrierTries; ++i) {
            if (*reinterpret_cast<volatile unsigned*>(count) >= target) {
                ok = 1;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Geodesic Voronoi labelling in one cooperative launch: every pass relaxes all tiles
// (block b takes tiles b, b + grid, ...), a grid barrier closes it, and the passes
// stop at the first that changed nothing (every block reads the same count after
// the barrier) or after kMaxPasses, which is recorded as a failure; so is a barrier
// that gave up. No host round trip between passes.
__global__ void __launch_bounds__(kThreads) epic_voronoi_kernel(const int* cost, unsigned long long* key, int W, int H,
                                                                int* changed, unsigned* sync_count, int* err)
{
    const int tiles_x = (W + kTile - 1) / kTile, n_tiles = tiles_x * ((H + kTile - 1) / kTile);
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0;
    for (int pass = 0; pass < kMaxPasses; ++pass) {
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x)
            voronoi_tile(cost, key, W, H, changed, pass, (t % tiles_x) * kTile, (t / tiles_x) * kTile);
        if (!grid_barrier(sync_count, (unsigned)(pass + 1) * gridDim.x)) {
            if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(err, kErrSync);
            return;
        }
        if (*reinterpret_cast<volatile int*>(changed + pass) == 0) return;
    }
    if (lead) atomicOr(err, kErrPasses);
}

// Records a device-side failure of the call in the library's status word.
__global__ void epic_report_kernel(const int* err, unsigned* status)
{
    const int e = *err;
    if (e && status) atomicOr(status, e & (kErrPasses | kErrSync) ? DGF_DEV_EPIC_PASSES : DGF_DEV_EPIC_CAPACITY);
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

// Multi-block exclusive scan of the link counts: each block scans 1024 counts and
// publishes its total; the one-block scan above turns the totals into block
// offsets; a last pass adds them (and fills the cursors).
__global__ void __launch_bounds__(1024) epic_scan_blocks_kernel(const int* cnt, int n, int* off, int* bsum)
{
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int i = blockIdx.x * 1024 + t;
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
    if (i < n) off[i] = (w ? wsum[w - 1] : 0) + x - v;
    if (t == 0) bsum[blockIdx.x] = wsum[31];
}

__global__ void __launch_bounds__(1024) epic_scan_add_kernel(const int* boff, int n, int nb, int* off, int* cur)
{
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n) {
        const int o = off[i] + boff[blockIdx.x];
        off[i] = o;
        cur[i] = o;
    }
    if (i == 0) off[n] = boff[nb];
}

// Per seed: keeps one link per neighbour (the smallest weight), compacting the list
// in place; end[s] becomes the end of the compacted list. One warp per seed walks
// the list in chunks of 32: lanes holding the same neighbour find each other with
// match.any and take their minimum weight; the lowest of them either lowers the
// weight of a link kept from an earlier chunk or appends a new one. The kept prefix
// never reaches the unread part of the list.
__global__ void __launch_bounds__(kThreads) epic_dedupe_kernel(const int* off, int* end, int* adj_t, long long* adj_w,
                                                               unsigned* minin, int n)
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
    // smallest link weight (a lower bound on the last step of any path into s),
    // clamped to 32 bits (a smaller bound stays a bound)
    long long mn = kNoLink;
    for (int j = b + lane; j < out; j += 32) mn = min(mn, adj_w[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) {
        end[s] = out;
        minin[s] = (unsigned)min(mn, (long long)kNoLink);
    }
}

// Link records for the search: (neighbour, its list begin, its list end, its
// smallest link weight).
__global__ void __launch_bounds__(kThreads) epic_link_meta_kernel(const int* off, const int* end, const int* adj_t,
                                                                  const unsigned* minin, int4* adj_i, int n)
{
    const int s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= n) return;
    for (int i = off[s], e = end[s]; i < e; ++i) {
        const int t = adj_t[i];
        adj_i[i] = make_int4(t, off[t], end[t], (int)minin[t]);
    }
}

struct KnnArgs {
    const float2* pts;
    const float2* flow;
    const int* seed_pix;
    const int* off;
    const int* end;
    const unsigned* minin;
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
    int n, k, model;
    double a_per_unit, min_spread2;  // kernel decay per unit of distance: a / (2 cost_base)
};

// Per-warp shared layout of one search: a hash of HCAP discovered seeds (index,
// tentative distance, smallest incoming link weight, settled flag), the frontier
// as a list of FCAP hash slots, and the settled keys (SCAP, later sorted in place).
template <int HCAP, int FCAP, int SCAP>
struct KnnLayout {
    static_assert(HCAP % 32 == 0 && (SCAP & (SCAP - 1)) == 0 && HCAP <= 32768, "sizes");
    static constexpr size_t o_hdist = (size_t)HCAP * 4;
    static constexpr size_t o_sort = o_hdist + (size_t)HCAP * 8;
    static constexpr size_t o_minin = o_sort + (size_t)SCAP * 8;
    static constexpr size_t o_front = o_minin + (size_t)HCAP * 4;
    static constexpr size_t o_state = o_front + (size_t)FCAP * 2;
    static constexpr size_t o_count = (o_state + (size_t)HCAP + 15) & ~(size_t)15;
    static constexpr size_t bytes = o_count + 16;
};

// The fast layouts hold every search of the benchmark scenes (at k = 128 at most
// about 250 discovered and 171 settled seeds, in a 384-slot hash; larger k takes
// the larger one); a search that outgrows them is redone by the retry kernel with
// room for 8192.
constexpr int kFastWarps = 4, kSmallK = 160;
constexpr int kBigH = 8192, kBigF = 8192, kBigS = 8192;  // the retry kernel runs one block per SM
constexpr int kRetry = 16;  // search status: capacity exceeded, redo with the large layout
constexpr long long kInf = 0x7fffffffffffffffll;
enum : unsigned char { kFrontier = 0, kSettled = 1 };

// exp(-y) for y >= 0 by the table-driven method of Tang (ACM TOMS 15(2), 1989):
// y = (32 q + j) ln2 / 32 + r with |r| <= ln2 / 64, so exp(-y) = 2^-q 2^(-j/32)
// exp(-r), exp(-r) by its degree-6 Taylor polynomial (truncation below 4e-18); the
// reduction uses a two-part ln2 / 32 and fused multiply-adds; the power of two is
// built from exponent bits. Within 2 ulps of the result (measured against an
// extended-precision exp: 1.93 ulps on normal results, 1.27 on subnormal ones); 0
// from y = 745.2 on, where exp(-y) is below half the smallest subnormal.
__device__ const double kExp2Frac[32] = {  // 2^(-j/32), correctly rounded
    0x1.0000000000000p+0, 0x1.f50765b6e4540p-1, 0x1.ea4afa2a490dap-1, 0x1.dfc97337b9b5fp-1,
    0x1.d5818dcfba487p-1, 0x1.cb720dcef9069p-1, 0x1.c199bdd85529cp-1, 0x1.b7f76f2fb5e47p-1,
    0x1.ae89f995ad3adp-1, 0x1.a5503b23e255dp-1, 0x1.9c49182a3f090p-1, 0x1.93737b0cdc5e5p-1,
    0x1.8ace5422aa0dbp-1, 0x1.82589994cce13p-1, 0x1.7a11473eb0187p-1, 0x1.71f75e8ec5f74p-1,
    0x1.6a09e667f3bcdp-1, 0x1.6247eb03a5585p-1, 0x1.5ab07dd485429p-1, 0x1.5342b569d4f82p-1,
    0x1.4bfdad5362a27p-1, 0x1.44e086061892dp-1, 0x1.3dea64c123422p-1, 0x1.371a7373aa9cbp-1,
    0x1.306fe0a31b715p-1, 0x1.29e9df51fdee1p-1, 0x1.2387a6e756238p-1, 0x1.1d4873168b9aap-1,
    0x1.172b83c7d517bp-1, 0x1.11301d0125b51p-1, 0x1.0b5586cf9890fp-1, 0x1.059b0d3158574p-1,
};

__device__ __forceinline__ double exp_neg(double y)
{
    if (!(y < 745.2)) return 0.0;
    const double kf = rint(y * 0x1.71547652b82fep+5);  // y * 32 / ln2
    double r = fma(-kf, 0x1.62e42fefa39efp-6, y);      // ln2 / 32, leading part
    r = fma(-kf, 0x1.abc9e3b39803fp-61, r);            // and the rest
    const double x = -r;
    double e = 1.0 / 720.0;
    e = fma(e, x, 1.0 / 120.0);
    e = fma(e, x, 1.0 / 24.0);
    e = fma(e, x, 1.0 / 6.0);
    e = fma(e, x, 0.5);
    e = fma(e, x, 1.0);
    e = fma(e, x, 1.0);
    const int k = (int)kf, q = k >> 5;  // q <= 1075: 2^-q as two normal powers of two
    const double s1 = __longlong_as_double((long long)(1023 - (q >> 1)) << 52);
    const double s2 = __longlong_as_double((long long)(1023 - (q - (q >> 1))) << 52);
    return e * __ldg(&kExp2Frac[k & 31]) * s1 * s2;
}

// Double-float arithmetic (an unevaluated pair hi + lo of FP32 values, about 48
// significant bits; Dekker 1971, Knuth's TwoSum): the fit's per-neighbour products
// and sums run on GB300's wide FP32 pipe instead of its narrow FP64 pipe, at an
// accuracy far inside what the fit needs. Written with the _rn intrinsics so that
// no addition is contracted or reordered.
struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b)  // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_mul(dfl a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const dfl s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfl to_dfl(double v)
{
    const float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

// Sums of 12 values over the warp; the totals land in lane 0. Halving exchanges:
// lanes 16 apart swap half of their values and keep the sum of the other half, then
// lanes 8 apart the same with 3 of 6, then xor butterflies finish the 3 sums in each
// group of 8 lanes; lanes 8, 16 and 24 hand their 3 totals to lane 0.
__device__ __forceinline__ void warp_sum12(const double (&v)[12], double (&out)[12])
{
    const int lane = threadIdx.x & 31;
    const bool hi16 = lane & 16, hi8 = lane & 8;
    double h[6], q[3];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double keep = hi16 ? v[6 + i] : v[i], give = hi16 ? v[i] : v[6 + i];
        h[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double keep = hi8 ? h[3 + i] : h[i], give = hi8 ? h[i] : h[3 + i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 3; ++i) q[i] += __shfl_xor_sync(0xffffffffu, q[i], o);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        out[i] = q[i];
        out[3 + i] = __shfl_sync(0xffffffffu, q[i], 8);
        out[6 + i] = __shfl_sync(0xffffffffu, q[i], 16);
        out[9 + i] = __shfl_sync(0xffffffffu, q[i], 24);
    }
}

__device__ __forceinline__ long long warp_min64(long long v)  // v >= 0
{
    const unsigned hi = __reduce_min_sync(0xffffffffu, (unsigned)((unsigned long long)v >> 32));
    const unsigned lo = __reduce_min_sync(0xffffffffu, (unsigned)((unsigned long long)v >> 32) == hi ? (unsigned)v : ~0u);
    return (long long)(((unsigned long long)hi << 32) | lo);
}

// Ascending bitonic sort of N keys (a power of two) in shared memory by one warp.
__device__ void warp_bitonic_sort(unsigned long long* key, int N)
{
    const int lane = threadIdx.x & 31;
    for (int size = 2; size <= N; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < N / 2; i += 32) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long x = key[lo], y = key[hi];
                if ((x > y) == asc) {
                    key[lo] = y;
                    key[hi] = x;
                }
            }
            __syncwarp();
        }
}

// The k nearest seeds of seed s in the seed graph, exactly, by Dijkstra with batch
// settling: with m the smallest tentative distance on the frontier, every frontier
// seed v with d(v) <= m + minin(v) is final (a shorter path would have to end with
// a link from an unsettled seed, at least m away, and that link weighs at least
// minin(v)); the whole batch is settled (appended to the settled keys and removed
// from the frontier list), then its links are relaxed, one lane per batch seed;
// newly discovered seeds join the frontier list. The search stops once k settled
// seeds lie below m (every unsettled seed is at least m away) or the frontier is
// empty; the settled keys (distance << 24 | index) are then sorted and the first
// k kept (cnt_out). Returns 0, kRetry when the hash, the frontier list or the
// settled list is full, or kErrRange when a distance leaves 40 bits.
template <int HCAP, int FCAP, int SCAP>
__device__ int knn_search(const KnnArgs& a, int s, unsigned char* base, int& cnt_out)
{
    using Lay = KnnLayout<HCAP, FCAP, SCAP>;
    int* hkey = reinterpret_cast<int*>(base);
    volatile int* vh = hkey;
    long long* hdist = reinterpret_cast<long long*>(base + Lay::o_hdist);
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(base + Lay::o_sort);
    unsigned* hmin = reinterpret_cast<unsigned*>(base + Lay::o_minin);
    short* front = reinterpret_cast<short*>(base + Lay::o_front);
    unsigned char* hst = base + Lay::o_state;
    int* fcount = reinterpret_cast<int*>(base + Lay::o_count);  // frontier list length
    const int lane = threadIdx.x & 31;
    // multiplicative hash scaled onto [0, HCAP) (HCAP need not be a power of two)
    auto slot_of = [](int t) {
        return (int)(((unsigned long long)((unsigned)t * 0x9E3779B1u) * (unsigned)HCAP) >> 32);
    };

    for (int j = lane; j < HCAP; j += 32) {
        hkey[j] = -1;
        hdist[j] = kInf;
        hst[j] = kFrontier;
    }
    __syncwarp();
    if (lane == 0) {
        const int h = slot_of(s);
        hkey[h] = s;
        hdist[h] = 0;
        hmin[h] = a.minin[s];
        front[0] = (short)h;
        *fcount = 1;
    }
    __syncwarp();
    int status = 0, nset = 0;
    for (int step = 0; step < HCAP; ++step) {  // every step settles at least the frontier minimum
        const int nf = *fcount;
        if (nf == 0) break;  // every reachable seed is settled
        long long m = kInf;
        for (int i = lane; i < nf; i += 32) m = min(m, hdist[front[i]]);
        m = warp_min64(m);
        int below = 0;
        for (int i = lane; i < nset; i += 32) below += (long long)(skey[i] >> kIdxBits) < m;
        if ((int)__reduce_add_sync(0xffffffffu, (unsigned)below) >= a.k) break;
        // settle the batch: compact the frontier list in place (chunks are read
        // before the kept entries of the chunk are written, and never ahead of them)
        const int nset0 = nset;
        int kept = 0;
        for (int c = 0; c < nf; c += 32) {
            const int i = c + lane;
            int h = -1;
            bool bat = false;
            if (i < nf) {
                h = front[i];
                bat = hdist[h] <= m + (long long)hmin[h];
            }
            const unsigned bm = __ballot_sync(0xffffffffu, bat), km = __ballot_sync(0xffffffffu, i < nf && !bat);
            const unsigned lt = (1u << lane) - 1;
            __syncwarp();
            if (bat) {
                const int pos = nset + __popc(bm & lt);
                if (pos < SCAP) {
                    skey[pos] = ((unsigned long long)hdist[h] << kIdxBits) | (unsigned long long)hkey[h];
                    hst[h] = kSettled;
                }
            } else if (i < nf) {
                front[kept + __popc(km & lt)] = (short)h;
            }
            nset += __popc(bm);
            kept += __popc(km);
            __syncwarp();
        }
        if (nset > SCAP) {
            status = kRetry;
            break;
        }
        if (lane == 0) *fcount = kept;
        __syncwarp();
        // relax the batch's links, one lane per link: the batch seeds' link counts
        // are prefix-summed over the warp (32 seeds at a time) and each lane finds
        // the seed owning its link by a binary search over the sums, so all the
        // links' loads are in flight together
        int st = 0;
        for (int b0 = nset0; b0 < nset; b0 += 32) {
            const int nb = min(32, nset - b0);
            int u = 0, first = 0, deg = 0;
            long long du = 0;
            if (lane < nb) {
                const unsigned long long kb = skey[b0 + lane];
                u = (int)(kb & kIdxMask);
                du = (long long)(kb >> kIdxBits);
                first = a.off[u];
                deg = a.end[u] - first;
            }
            int incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int c0 = 0; c0 < total; c0 += 32) {
                const int e = c0 + lane;
                // owner: the first batch lane whose inclusive sum exceeds e
                int lo = 0, hi = nb - 1;
#pragma unroll
                for (int it = 0; it < 5; ++it) {
                    const int mid = (lo + hi) >> 1;
                    const int v = __shfl_sync(0xffffffffu, incl, mid);
                    if (v > e) hi = mid; else lo = min(mid + 1, hi);
                }
                const int ow = lo;
                const int ofirst = __shfl_sync(0xffffffffu, first, ow);
                const int oexcl = __shfl_sync(0xffffffffu, incl - deg, ow);
                const long long odu = __shfl_sync(0xffffffffu, du, ow);
                if (e >= total || st) continue;
                const int le = ofirst + (e - oexcl);
                const int4 li = a.adj_i[le];
                const long long nd = odu + a.adj_w[le];
                if (nd >= kDistLimit) st |= kErrRange;
                const int t = li.x;
                int h = slot_of(t), hs = -1;
                for (int q = 0; q < HCAP; ++q) {
                    const int c = vh[h];
                    if (c == t) {
                        hs = h;
                        break;
                    }
                    if (c == -1) {
                        const int prev = atomicCAS(&hkey[h], -1, t);
                        if (prev == -1) {  // discovered: joins the frontier list
                            hmin[h] = (unsigned)li.w;
                            const int f = atomicAdd(fcount, 1);
                            if (f < FCAP)
                                front[f] = (short)h;
                            else
                                st |= kRetry;
                            hs = h;
                            break;
                        }
                        if (prev == t) {
                            hs = h;
                            break;
                        }
                    }
                    h = h + 1 == HCAP ? 0 : h + 1;
                }
                if (hs < 0) {
                    st |= kRetry;
                    continue;
                }
                // a settled seed keeps its final distance: the minimum is a no-op there
                if (hst[hs] == kFrontier)
                    atomicMin(reinterpret_cast<unsigned long long*>(&hdist[hs]), (unsigned long long)nd);
            }
        }
        __syncwarp();
        status = __reduce_or_sync(0xffffffffu, st);
        if (status) break;
    }
    if (!status) {
        int N = 32;
        while (N < nset) N <<= 1;
        if (N > SCAP) {
            status = kRetry;
        } else {
            for (int j = nset + lane; j < N; j += 32) skey[j] = kNone;
            __syncwarp();
            warp_bitonic_sort(skey, N);
            cnt_out = min(nset, a.k);
        }
    }
    return status & kErrRange ? kErrRange : status;
}

// The weighted affine fit of seed s over its neighbourhood (sorted keys) and the
// outputs. The 3 x 3 normal equations lose too many digits in FP32 when a
// neighbourhood is narrow: the weights come from an FP64 exponential, the
// per-neighbour terms are summed in double-float, the lanes' sums are reduced and
// the systems solved in FP64. M = sum w v v^T, v = (x_t - x_s, y_t - y_s, 1).
__device__ void knn_fit_write(const KnnArgs& a, int s, int cnt, const unsigned long long* key)
{
    const int lane = threadIdx.x & 31, k = a.k;
    if (a.knn_count && lane == 0) a.knn_count[s] = cnt;
    if (a.knn_idx)
        for (int j = lane; j < cnt; j += 32) {
            a.knn_idx[(size_t)s * k + j] = (int)(key[j] & kIdxMask);
            a.knn_dist[(size_t)s * k + j] = (int64_t)(key[j] >> kIdxBits);
        }
    const float2 ps = a.pts[s];
    dfl acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
    for (int j = lane; j < cnt; j += 32) {
        const int t = (int)(key[j] & kIdxMask);
        const dfl w = to_dfl(exp_neg(a.a_per_unit * (double)(long long)(key[j] >> kIdxBits)));
        const float2 pt = a.pts[t], ft = a.flow[t];
        const dfl vx = two_sum(pt.x, -ps.x), vy = two_sum(pt.y, -ps.y);  // exact differences
        const dfl wx = df_mul(w, vx), wy = df_mul(w, vy);
        acc[0] = df_add(acc[0], df_mul(wx, vx));
        acc[1] = df_add(acc[1], df_mul(wx, vy));
        acc[2] = df_add(acc[2], wx);
        acc[3] = df_add(acc[3], df_mul(wy, vy));
        acc[4] = df_add(acc[4], wy);
        acc[5] = df_add(acc[5], w);
        acc[6] = df_add(acc[6], df_mul(wx, ft.x));
        acc[7] = df_add(acc[7], df_mul(wy, ft.x));
        acc[8] = df_add(acc[8], df_mul(w, ft.x));
        acc[9] = df_add(acc[9], df_mul(wx, ft.y));
        acc[10] = df_add(acc[10], df_mul(wy, ft.y));
        acc[11] = df_add(acc[11], df_mul(w, ft.y));
    }
    double accd[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) accd[i] = (double)acc[i].hi + (double)acc[i].lo;
    double tot[12];
    warp_sum12(accd, tot);
    if (lane != 0) return;
    const double m00 = tot[0], m01 = tot[1], m02 = tot[2], m11 = tot[3], m12 = tot[4], m22 = tot[5];
    const double u0 = tot[6], u1 = tot[7], u2 = tot[8], v0 = tot[9], v1 = tot[10], v2 = tot[11];
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

// One warp per seed with a fast layout; searches that outgrow it are queued for
// the retry kernel.
template <int HCAP, int FCAP, int SCAP>
__global__ void __launch_bounds__(kFastWarps * 32) epic_knn_fit_kernel(KnnArgs a)
{
    using Lay = KnnLayout<HCAP, FCAP, SCAP>;
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
    unsigned char* base = smem + (size_t)wid * Lay::bytes;
    int cnt = 0;
    const int st = knn_search<HCAP, FCAP, SCAP>(a, s, base, cnt);
    if (st == kRetry) {
        if (lane == 0) a.retry_list[atomicAdd(a.retry_count, 1)] = s;
        return;
    }
    if (st) {
        if (lane == 0) atomicOr(a.err, st);
        return;
    }
    knn_fit_write(a, s, cnt, reinterpret_cast<const unsigned long long*>(base + Lay::o_sort));
}

// The queued searches with room for 8192 discovered seeds, one warp per block.
__global__ void __launch_bounds__(32) epic_knn_retry_kernel(KnnArgs a)
{
    using Lay = KnnLayout<kBigH, kBigF, kBigS>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int total = *a.retry_count;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        const int s = a.retry_list[i];
        int cnt = 0;
        const int st = knn_search<kBigH, kBigF, kBigS>(a, s, smem, cnt);
        if (st) {
            if ((threadIdx.x & 31) == 0) atomicOr(a.err, st == kRetry ? kErrFrontier : st);
            continue;
        }
        knn_fit_write(a, s, cnt, reinterpret_cast<const unsigned long long*>(smem + Lay::o_sort));
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
    size_t key, cost, seed_pix, cnt, off, cur, minin, bsum, adj_t, adj_w, adj_i, models, retry, counters, total;
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
    L.minin = take((size_t)n * 4);
    L.bsum = take(((size_t)n / 1024 + 2) * 12);  // block totals, block offsets (+1), scan cursors
    L.adj_t = take(nl * 4);
    L.adj_w = take(nl * 8);
    L.adj_i = take(nl * 16);
    L.models = take((size_t)n * 48);
    L.retry = take((size_t)n * 4);
    L.counters = take((kMaxPasses + 3) * 4);  // pass counters, the status word, the retry count, the barrier
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

namespace {

__global__ void exp_neg_kernel(const double* y, double* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = exp_neg(y[i]);
}

}  // namespace

// The exponential of the fit weights, exported so that its accuracy can be checked
// against a reference exp on the same arguments.
extern "C" int dgf_epic_exp_neg(const double* y, double* out, int n, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && (!y || !out))) return DGF_ERR_ARG;
    if (n == 0) return DGF_OK;
    exp_neg_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(y, out, n);
    return dgf::launch_status();
}

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
    auto* minin = reinterpret_cast<unsigned*>(ws + L.minin);
    auto* bsum = reinterpret_cast<int*>(ws + L.bsum);
    auto* retry_list = reinterpret_cast<int*>(ws + L.retry);
    auto* models = reinterpret_cast<double*>(ws + L.models);
    auto* changed = reinterpret_cast<int*>(ws + L.counters);
    int* err = changed + kMaxPasses;
    int* retry_count = err + 1;
    unsigned* sync_count = reinterpret_cast<unsigned*>(retry_count + 1);
    const float2* p2 = reinterpret_cast<const float2*>(pts);
    const float2* f2 = reinterpret_cast<const float2*>(flow);

    unsigned* dev_status = dgf::status_word();
    if (!dev_status) return DGF_ERR_CUDA;
    if (cudaMemsetAsync(changed, 0, (kMaxPasses + 3) * sizeof(int), stream) != cudaSuccess) return DGF_ERR_CUDA;
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

    // geodesic Voronoi labelling: passes until one changes nothing, in one
    // cooperative launch of as many blocks as can be resident (at most one a tile)
    {
        int per_sm = 0, dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, epic_voronoi_kernel, kThreads, 0) != cudaSuccess ||
            per_sm < 1)
            return DGF_ERR_CUDA;
        const long long tiles = (long long)((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
        const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)per_sm * sms);
        const dim3 block(32, 8);
        void* args[] = {(void*)&cost, (void*)&key, (void*)&W, (void*)&H, (void*)&changed, (void*)&sync_count,
                        (void*)&err};
        if (cudaLaunchCooperativeKernel((const void*)epic_voronoi_kernel, dim3(grid), block, args, 0, stream) !=
            cudaSuccess)
            return DGF_ERR_CUDA;
    }

    if (n > 0) {
        epic_links_kernel<false><<<pix_grid, pix_block, 0, stream>>>(key, cost, W, H, cnt, nullptr, nullptr, nullptr,
                                                                     nullptr, err);
        const int nb = (n + 1023) / 1024;
        epic_scan_blocks_kernel<<<nb, 1024, 0, stream>>>(cnt, n, off, bsum);
        epic_scan_kernel<<<1, 1024, 0, stream>>>(bsum, nb, bsum + nb, bsum + 2 * nb + 1);
        epic_scan_add_kernel<<<nb, 1024, 0, stream>>>(bsum + nb, n, nb, off, cur);
        epic_links_kernel<true><<<pix_grid, pix_block, 0, stream>>>(key, cost, W, H, nullptr, off, cur, adj_t, adj_w,
                                                                    err);
        epic_dedupe_kernel<<<(unsigned)((n + kThreads / 32 - 1) / (kThreads / 32)), kThreads, 0, stream>>>(
            off, cur, adj_t, adj_w, minin, n);
        epic_link_meta_kernel<<<pt_grid, kThreads, 0, stream>>>(off, cur, adj_t, minin, adj_i, n);
        KnnArgs a;
        a.pts = p2;
        a.flow = f2;
        a.seed_pix = seed_pix;
        a.off = off;
        a.end = cur;
        a.minin = minin;
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
        a.a_per_unit = p->a / (2.0 * p->cost_base);
        a.min_spread2 = p->min_spread * p->min_spread;
        const bool small = p->k <= kSmallK;
        auto fast = small ? epic_knn_fit_kernel<384, 256, 256> : epic_knn_fit_kernel<1024, 512, 512>;
        const size_t smem_fast =
            (small ? KnnLayout<384, 256, 256>::bytes : KnnLayout<1024, 512, 512>::bytes) * kFastWarps;
        const size_t smem_big = KnnLayout<kBigH, kBigF, kBigS>::bytes;
        if (cudaFuncSetAttribute(fast, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fast) != cudaSuccess ||
            cudaFuncSetAttribute(epic_knn_retry_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_big) !=
                cudaSuccess)
            return DGF_ERR_CUDA;
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return DGF_ERR_CUDA;
        fast<<<(unsigned)((n + kFastWarps - 1) / kFastWarps), kFastWarps * 32, smem_fast, stream>>>(a);
        epic_knn_retry_kernel<<<(unsigned)sms, 32, smem_big, stream>>>(a);
    }
    epic_dense_kernel<<<pix_grid, pix_block, 0, stream>>>(key, models, p2, W, H, reinterpret_cast<float2*>(dense),
                                                          d.labels, d.dist);
    if (d.retried &&
        cudaMemcpyAsync(d.retried, retry_count, sizeof(int), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return DGF_ERR_CUDA;
    epic_report_kernel<<<1, 1, 0, stream>>>(err, dev_status);
    return dgf::launch_status();
}
