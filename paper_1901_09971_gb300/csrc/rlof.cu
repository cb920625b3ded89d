// RLOF sparse point tracking (arXiv 1901.09971, Section 2 "Sparse point tracking";
// Section 3 "Parameters": RLOF with the illumination model).
//
// Work mapping: a group of G consecutive lanes (G = 8, 16 or 32) owns one point
// for its whole coarse-to-fine trajectory. The (2r+1)^2 support is cut into
// sample pairs that share the bilinear weights of the iterate and four of their
// six taps, so a pair is sampled with four loads and evaluated with packed FP32x2
// instructions (fma.rn.f32x2 and friends on sm_100+). For radius 4 and 5 the
// first 2r columns form horizontal pairs and the last column vertical ones (radius
// 5: 61 pairs, four slots of 16 lanes); other radii use (2r+1) x (r+1) horizontal
// pairs whose last column's second sample is masked out. Lane l of a group owns
// pairs l, l + G, l + 2G, ..., except at 8 lanes (the default for radius 4 and 5),
// where each lane owns two vertical runs of horizontal pairs whose tap rows are
// shared along the run (RunLayout) and one vertical pair.
//
// The template T, Tx, Ty of the current level is sampled once per level into
// shared memory (one 16-byte and one 8-byte slot per pair, read back without
// bank conflicts), which leaves the registers to the accumulators and the taps in
// flight. Per iteration every lane forms Hampel weights and its partial sums of
// the 4x4 (or 2x2) normal equations; the group reduces the 4x4 sums through a
// per-warp shared-memory scratch (bit-identical totals in every lane), and the
// FP32 solve, the update and the convergence test run redundantly, so each
// group's control flow stays uniform and points converge and exit independently.
//
// Time per iteration splits roughly 70% per-sample accumulation, 18% group
// reduction, 5% solve: the kernel is bound by instruction issue and dependency
// latency on the FP32 and integer pipes, not by memory (the pyramids stay in L1/L2).
#include <atomic>

#include "common.cuh"
#include "batch.cuh"

namespace rlof_detail {

using dgf::TrackBatch;

// Threads per block: 128 (eight points at 16 lanes) or, at 8 lanes, 32. A block's
// registers and warp slots are released only when its last warp ends, so small
// blocks free the slots of finished points sooner; measured on GB300, 32-thread
// blocks are 3% faster on the 64-pair batch (8 lanes) and 1.6% slower on the
// radius-5 driving-scene pair (16 lanes), where 128 stays.
template <int G>
__host__ __device__ constexpr int block_threads()
{
    return G == 8 ? 32 : 128;
}

// Resident blocks the register budget is sized for: 512 threads a SM (128 registers
// a thread), except at 8 lanes and radius 5, where the bound of 14 one-warp blocks
// gives the fastest code (128 registers, so 16 blocks fit; 4 bytes of spills, which
// the bounds of 15 and 16 avoid, measured 1.055 against 1.064 and 1.073 ms on the
// 1242x375 pair; before the offset was folded into the interpolation: 12, 13, 14 and
// 16 blocks 1.096, 1.080, 1.067 and 1.096 ms), and 12 for the cross-based support
// there (at 14 its arm scan spills).
template <int G, int RC, bool CROSS>
__host__ __device__ constexpr int min_blocks()
{
    if (G == 8 && RC == 5) return CROSS ? 12 : 14;
    return 512 / block_threads<G>();
}

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Per-warp scratch of the group reduction: one row of 16 partial sums per lane and
// 16 totals per group. Rows are 20 floats apart, so the 16-byte accesses of eight
// consecutive lanes start in distinct quads of banks.
constexpr int kRowStride = 20;
struct alignas(16) WarpScratch {
    float rows[32 * kRowStride];
    float totals[4 * 16];
};

__device__ __forceinline__ float4 add4(float4 a, float4 b)
{
    const float2 lo = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 hi = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Sum of 16 values over a group of G lanes, returned in every lane (h[k] = total of
// v[k] over the group). Every lane stores its values as a row; lane l adds value
// block l & 3 (values 4 (l & 3) .. +3) over the four rows 4 (l >> 2) .. +3 of its
// group; the G / 4 lanes holding the same block combine their partial sums with
// xor shuffles; lanes 0..3 publish the four block totals, which every lane of the
// group then reads back, so all lanes receive the same bits. Groups of a warp use
// disjoint rows and totals, so diverged groups never meet at a barrier.
template <int G>
__device__ __forceinline__ void group_allreduce16(const float (&v)[16], float (&h)[16], unsigned mask, int lane,
                                                  WarpScratch& ws)
{
    const int wl = threadIdx.x & 31;
    const int g0 = wl - lane;  // warp lane of the group's lane 0
    float4* row = reinterpret_cast<float4*>(ws.rows + wl * kRowStride);
#pragma unroll
    for (int i = 0; i < 4; ++i) row[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    __syncwarp(mask);
    const int blk = lane & 3;
    const float* src = ws.rows + (g0 + 4 * (lane >> 2)) * kRowStride + 4 * blk;
    float4 s = *reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 1; i < 4; ++i) s = add4(s, *reinterpret_cast<const float4*>(src + i * kRowStride));
#pragma unroll
    for (int o = 4; o < G; o <<= 1) {
        float4 t;
        t.x = __shfl_xor_sync(mask, s.x, o);
        t.y = __shfl_xor_sync(mask, s.y, o);
        t.z = __shfl_xor_sync(mask, s.z, o);
        t.w = __shfl_xor_sync(mask, s.w, o);
        s = add4(s, t);
    }
    float4* tot = reinterpret_cast<float4*>(ws.totals + (g0 / G) * 16);
    if (lane < 4) tot[blk] = s;
    __syncwarp(mask);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 t = tot[i];
        h[4 * i] = t.x;
        h[4 * i + 1] = t.y;
        h[4 * i + 2] = t.z;
        h[4 * i + 3] = t.w;
    }
    // ordering across calls: each lane reads the rows before the second
    // __syncwarp above, which precedes the next call's row stores, and reads the
    // totals before the next call's first __syncwarp, which precedes their rewrite
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Bilinear weights of the four taps (top-left, top-right, bottom-left,
// bottom-right) for fractional offsets (ax, ay), duplicated for a sample pair.
struct PairWeights {
    float2 w00, w01, w10, w11;
    __device__ __forceinline__ PairWeights(float ax, float ay)
    {
        const float bx = 1.f - ax, by = 1.f - ay;
        w00 = f2(bx * by);
        w01 = f2(ax * by);
        w10 = f2(bx * ay);
        w11 = f2(ax * ay);
    }
};

// Two horizontally adjacent bilinear samples from their 2x3 taps (a0 a1 a2 / b0 b1 b2).
__device__ __forceinline__ float2 bilinear_pair(const PairWeights& w, float a0, float a1, float a2, float b0,
                                                float b1, float b2)
{
    float2 J = __fmul2_rn(w.w00, make_float2(a0, a1));
    J = __ffma2_rn(w.w01, make_float2(a1, a2), J);
    J = __ffma2_rn(w.w10, make_float2(b0, b1), J);
    return __ffma2_rn(w.w11, make_float2(b1, b2), J);
}

// Loads of two consecutive samples starting at p; 8-byte aligned when requested.
__device__ __forceinline__ float2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ float2 ld2(const __half* p)
{
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
}

// Sample pair at integer tap origin (xi, yi) with every tap clamped to the border.
template <typename TS>
__device__ __forceinline__ float2 pair_clamped(const TS* P, int pitch, int W, int H, int xi, int yi,
                                               const PairWeights& w)
{
    const int xa = min(max(xi, 0), W - 1), xb = min(max(xi + 1, 0), W - 1), xc = min(max(xi + 2, 0), W - 1);
    const TS* r0 = P + (size_t)min(max(yi, 0), H - 1) * pitch;
    const TS* r1 = P + (size_t)min(max(yi + 1, 0), H - 1) * pitch;
    return bilinear_pair(w, dgf::ld(r0 + xa), dgf::ld(r0 + xb), dgf::ld(r0 + xc), dgf::ld(r1 + xa),
                         dgf::ld(r1 + xb), dgf::ld(r1 + xc));
}

// Two vertically adjacent bilinear samples from their 3x2 taps (a0 a1 / b0 b1 / c0 c1).
__device__ __forceinline__ float2 bilinear_vpair(const PairWeights& w, float a0, float a1, float b0, float b1,
                                                 float c0, float c1)
{
    float2 J = __fmul2_rn(w.w00, make_float2(a0, b0));
    J = __ffma2_rn(w.w01, make_float2(a1, b1), J);
    J = __ffma2_rn(w.w10, make_float2(b0, c0), J);
    return __ffma2_rn(w.w11, make_float2(b1, c1), J);
}

// Vertical sample pair at integer tap origin (xi, yi) with every tap clamped.
template <typename TS>
__device__ __forceinline__ float2 vpair_clamped(const TS* P, int pitch, int W, int H, int xi, int yi,
                                                const PairWeights& w)
{
    const int xa = min(max(xi, 0), W - 1), xb = min(max(xi + 1, 0), W - 1);
    const TS* r0 = P + (size_t)min(max(yi, 0), H - 1) * pitch;
    const TS* r1 = P + (size_t)min(max(yi + 1, 0), H - 1) * pitch;
    const TS* r2 = P + (size_t)min(max(yi + 2, 0), H - 1) * pitch;
    return bilinear_vpair(w, dgf::ld(r0 + xa), dgf::ld(r0 + xb), dgf::ld(r1 + xa), dgf::ld(r1 + xb), dgf::ld(r2 + xa),
                          dgf::ld(r2 + xb));
}

// The taps of one point's support at integer origin (bx, by) of a plane, read
// without clamping (the pyramid planes carry a replicated border wide enough for
// any support around a position inside the level). One code path serves both
// parities e of the first column, so the two points of a warp never split into two
// load sequences run one after the other: for a horizontal pair at element offset
// off, the aligned pair load u holds (a0, a1) when e = 0 and (a1, a2) when e = 1,
// the scalar s the remaining tap (a2 or a0), and the bilinear weights swap with the
// parity instead of the taps: J = wP u + wQ Q (+ the row below), Q = (a1, a2) or
// (a0, a1). A generic slot holds a horizontal or a vertical pair: sample A's four
// taps, then the two taps sample B adds at stored offsets (right column or row
// below).
template <typename TS>
struct TapBlock {
    const TS *base, *base_u, *base_s;
    int pitch, e;
    float2 wP, wQ, wPb, wQb;
    __device__ __forceinline__ TapBlock(const TS* plane, int pitch_, int bx, int by, const PairWeights& pw)
    {
        pitch = pitch_;
        base = plane + (ptrdiff_t)by * pitch + bx;
        e = bx & 1;
        base_u = base + e;
        base_s = base + (2 - 2 * e);
        wP = e ? pw.w01 : pw.w00;
        wQ = e ? pw.w00 : pw.w01;
        wPb = e ? pw.w11 : pw.w10;
        wQb = e ? pw.w10 : pw.w11;
    }
    // The interpolated pair plus init (a Gauss-Newton step passes -c, the offset of
    // the illumination model, so that its residual needs one instruction less; the
    // level set-up passes 0).
    __device__ __forceinline__ float2 pair(int off, float2 init = make_float2(0.f, 0.f)) const
    {
        const TS* pu = base_u + off;
        const TS* ps = base_s + off;
        const float2 u = ld2(pu), ub = ld2(pu + pitch);
        const float sa = dgf::ld(ps), sb = dgf::ld(ps + pitch);
        const float2 Q = make_float2(e ? sa : u.y, e ? u.x : sa);
        const float2 Qb = make_float2(e ? sb : ub.y, e ? ub.x : sb);
        float2 J = __ffma2_rn(wP, u, init);
        J = __ffma2_rn(wQ, Q, J);
        J = __ffma2_rn(wPb, ub, J);
        return __ffma2_rn(wQb, Qb, J);
    }
    // One tap row of a horizontal pair, read at element offset k rows below the
    // run's first row (pu, ps: base_u, base_s plus the run's offset): the aligned
    // pair u and the pair Q the parity completes. pair_rows evaluates the pair whose
    // top and bottom tap rows these are, in the same order of operations as pair().
    struct Row {
        float2 u, Q;
    };
    __device__ __forceinline__ Row row(const TS* pu, const TS* ps, int k) const
    {
        const float2 u = ld2(pu + k * pitch);
        const float s = dgf::ld(ps + k * pitch);
        return Row{u, make_float2(e ? s : u.y, e ? u.x : s)};
    }
    __device__ __forceinline__ float2 pair_rows(const Row& t, const Row& b, float2 init) const
    {
        float2 J = __ffma2_rn(wP, t.u, init);
        J = __ffma2_rn(wQ, t.Q, J);
        J = __ffma2_rn(wPb, b.u, J);
        return __ffma2_rn(wQb, b.Q, J);
    }
    __device__ __forceinline__ float2 generic(int off, int eo0, int eo1, bool vert, const PairWeights& pw,
                                              float2 init = make_float2(0.f, 0.f)) const
    {
        const TS* p = base + off;
        const float a0 = dgf::ld(p), a1 = dgf::ld(p + 1), b0 = dgf::ld(p + pitch), b1 = dgf::ld(p + pitch + 1);
        const float e0 = dgf::ld(base + eo0), e1 = dgf::ld(base + eo1);
        const float t0 = vert ? b0 : a1, t1 = vert ? b1 : e0, t2 = vert ? e0 : b1;
        float2 J = __ffma2_rn(pw.w00, make_float2(a0, t0), init);
        J = __ffma2_rn(pw.w01, make_float2(a1, t1), J);
        J = __ffma2_rn(pw.w10, make_float2(b0, t2), J);
        return __ffma2_rn(pw.w11, make_float2(b1, e1), J);
    }
};

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Hampel IRLS weight psi(r) / r of the continuous three-part Hampel function:
//   min(1, a / |r|) * clamp((c - |r|) / (c - b), 0, 1)
// equals 1 for |r| <= a, a / |r| up to b, a (c - |r|) / ((c - b) |r|) up to c, 0 beyond.
__device__ __forceinline__ float hampel_weight(float r, float ha, float icb, float hc_icb)
{
    const float ar = fabsf(r);
    const float w = __saturatef(ha * rcp_approx(ar));
    return w * __saturatef(fmaf(-ar, icb, hc_icb));
}

__device__ __forceinline__ float rcp_approx_denorm(float x)
{
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Solve of the symmetric positive definite 4 x 4 system [[A, B], [B^T, C]] x = r
// (2 x 2 blocks) by block elimination: with the Schur complement S = C - B^T A^-1 B,
// x1 = S^-1 (r1 - B^T A^-1 r0) and x0 = A^-1 r0 - (A^-1 B) x1, the 2 x 2 inverses
// taken from their adjugates. The Cholesky pivots are a00, det A / a00, s00 and
// det S / s00, so the positivity test is the same as Cholesky's; returns false on
// failure. Its dependency chain is shorter than the sequential factorisation's.
__device__ __forceinline__ bool block_solve4(const float (&H)[4][4], const float (&r)[4], float (&x)[4])
{
    const float a00 = H[0][0], a01 = H[0][1], a11 = H[1][1];
    const float dA = fmaf(a00, a11, -a01 * a01);
    if (!(a00 > 0.f) || !(dA > 0.f)) return false;
    const float iA = rcp_approx_denorm(dA);
    const float i00 = a11 * iA, i01 = -a01 * iA, i11 = a00 * iA;  // A^-1
    const float b00 = H[0][2], b01 = H[0][3], b10 = H[1][2], b11 = H[1][3];
    const float x00 = fmaf(i00, b00, i01 * b10), x01 = fmaf(i00, b01, i01 * b11);  // X = A^-1 B
    const float x10 = fmaf(i01, b00, i11 * b10), x11 = fmaf(i01, b01, i11 * b11);
    const float s00 = H[2][2] - fmaf(b00, x00, b10 * x10);  // S = C - B^T X
    const float s01 = H[2][3] - fmaf(b00, x01, b10 * x11);
    const float s11 = H[3][3] - fmaf(b01, x01, b11 * x11);
    const float dS = fmaf(s00, s11, -s01 * s01);
    if (!(s00 > 0.f) || !(dS > 0.f)) return false;
    const float iS = rcp_approx_denorm(dS);
    const float y0 = fmaf(i00, r[0], i01 * r[1]), y1 = fmaf(i01, r[0], i11 * r[1]);  // A^-1 r0
    const float t0 = r[2] - fmaf(b00, y0, b10 * y1), t1 = r[3] - fmaf(b01, y0, b11 * y1);
    x[2] = fmaf(s11, t0, -s01 * t1) * iS;
    x[3] = fmaf(s00, t1, -s01 * t0) * iS;
    x[0] = y0 - fmaf(x00, x[2], x01 * x[3]);
    x[1] = y1 - fmaf(x10, x[2], x11 * x[3]);
    return true;
}

// Cholesky solve of the symmetric positive definite N x N system H x = rhs.
// Returns false on a non-positive pivot.
template <int N>
__device__ __forceinline__ bool chol_solve(float (&H)[N][N], const float (&rhs)[N], float (&x)[N])
{
    float L[N][N];
    float inv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float s = H[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fmaf(-L[i][k], L[j][k], s);
            if (i == j) {
                if (!(s > 0.f)) return false;
                inv[i] = rsqrtf(s);
                L[i][i] = s * inv[i];
            } else {
                L[i][j] = s * inv[j];
            }
        }
    }
    float z[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float s = rhs[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s = fmaf(-L[i][k], z[k], s);
        z[i] = s * inv[i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        float s = z[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) s = fmaf(-L[k][i], x[k], s);
        x[i] = s * inv[i];
    }
    return true;
}

// Support layouts. Runtime radius R: (2R+1) x (R+1) horizontal sample pairs, the
// second sample of each row's last pair masked out. Compile-time radius RC (4, 5):
// the first 2RC columns form (2RC+1) x RC horizontal pairs and the last column
// RC + 1 vertical pairs (rows 2k, 2k+1; the last one's second sample masked out),
// 2RC^2 + 2RC + 1 pairs in all, so 16 lanes cover radius 5 in 4 pair slots
// instead of 5. Pairs are numbered horizontal first; lane l owns l, l + G, ...
template <int RC>
struct Layout {
    static constexpr int side = 2 * RC + 1;
    static constexpr int nh = side * RC;     // horizontal pairs
    static constexpr int np = nh + RC + 1;   // all pairs
};

// Run layout (8 lanes, radius 4 and 5): the horizontal pairs of the first 2RC
// columns are grouped into vertical runs of pairs in one two-column strip; the
// pairs of a run share their tap rows, so a run of n pairs reads n + 1 rows of taps
// instead of 2n. Every lane owns two runs (slots 0 .. la - 1 and la .. la + lb - 1),
// then generic slots. A pair past the support is a pad: zero template, zero weight.
// Pads are whole runs at radius 5 (reading run 0's taps) and the last pair of a run
// at radius 4 (reading one row below the tap block, inside the planes' replicated
// border).
// * Radius 5 (11 pair rows, five strips), runs of 3: run t = lane + 8k covers strip
//   t % 5, pair rows 3 (t / 5) .. + 2 (15 runs; lane 7's second run is a pad); the
//   generic slots hold the pairs of rows 9 and 10 (g = lane + 8 (j - 6) < 10) and
//   the six vertical pairs of the last column (g >= 10).
// * Radius 4 (9 pair rows, four strips), a run of 2 and one of 3: strip s holds rows
//   0-1 (short run of lane s), 2-4 (long run of lane s), 5-6 (short run of lane
//   s + 4) and 7-9 (long run of lane s + 4, row 9 a pad); the generic slot holds
//   the five vertical pairs of the last column (g = lane).
// Measured on GB300 against each other: the radius-5 pair, 1.068 ms with runs of 3
// against 1.090 with runs of 3 and 4 plus a vertical slot; the radius-4 batch
// pair, 0.627 ms with runs of 2 and 3 against 0.647 with two runs of 2.
template <int G, int RC>
struct RunLayout {
    static constexpr bool on = G == 8 && (RC == 4 || RC == 5);
    static constexpr int la = RC == 5 ? 3 : 2;  // pairs of a lane's first run
    static constexpr int lb = 3;                // pairs of its second run
    static constexpr int first_generic = la + lb;
    static constexpr int nhg = RC == 5 ? 10 : 0;  // horizontal pairs in generic slots
    static constexpr int ng = nhg + RC + 1;       // generic pairs (then the vertical ones)
    static constexpr int slots = first_generic + (ng + G - 1) / G;
};

// Strip and first pair row of run k of a lane in the radius-4 run layout.
__device__ __forceinline__ void run_origin4(int lane, int k, int& strip, int& row)
{
    strip = lane & 3;
    row = k == 0 ? (lane < 4 ? 0 : 5) : (lane < 4 ? 2 : 7);
}

// Tap origin (x, y) in the support of sample A of slot j of a lane, whether the
// pair is vertical, and whether the slot holds a pair of the support (false for
// pads and slots past the support; their template is zeroed).
template <int G, int RC>
__device__ __forceinline__ bool slot_origin(int lane, int j, int R, int& x, int& y, bool& vert)
{
    vert = false;
    if constexpr (RunLayout<G, RC>::on) {
        using RL = RunLayout<G, RC>;
        if (j < RL::first_generic && RC == 5) {
            const int t = lane + G * (j / RL::la);  // run index
            const int tt = t < 15 ? t : 0;          // a pad run reads run 0's taps
            x = 2 * (tt % RC);
            y = RL::la * (tt / RC) + j % RL::la;
            return t < 15;
        }
        if (j < RL::first_generic) {
            const int k = j < RL::la ? 0 : 1;
            int strip, row;
            run_origin4(lane, k, strip, row);
            x = 2 * strip;
            y = row + (k ? j - RL::la : j);
            return y < 2 * RC + 1;
        }
        const int g = lane + G * (j - RL::first_generic);
        if (g < RL::nhg) {
            x = 2 * (g % RC);
            y = 9 + g / RC;
        } else {
            vert = true;
            x = 2 * RC;
            y = 2 * (g - RL::nhg);
        }
        return g < RL::ng;
    } else {
        const int pc = R + 1, np = RC ? Layout<RC>::np : (2 * R + 1) * pc;
        const int q = lane + G * j;
        if constexpr (RC == 0) {
            y = q / pc;
            x = 2 * (q - y * pc);
        } else if (q < Layout<RC>::nh) {
            y = q / RC;
            x = 2 * (q - y * RC);
        } else {
            vert = true;
            x = 2 * RC;
            y = 2 * (q - Layout<RC>::nh);
        }
        return q < np;
    }
}

// Per-lane state of one point's support at the current level: the template
// T, Tx, Ty of each owned pair (in shared memory: (T, Tx) of slot j at tq[32 j],
// Ty at ty[32 j], so a warp's 16- and 8-byte accesses are conflict-free), the
// pair's tap offset in the tap block and the mask of its second sample (0 where
// it lies past the support). Slots that can hold vertical pairs (compile-time
// layout only; at most the last two) also keep the offsets of the two taps the
// second sample adds, and a bit per such slot set for a vertical pair. In the run
// layout, each run's first tap row offset and a 0/1 factor on the weights of the
// pairs that can be pads (0 for a pad); last_ok is false when the lane's last slot
// lies past the support.
template <int SLP>
struct Support {
    float4* tq;
    float2* ty;
    __device__ __forceinline__ void put(int j, float2 T, float2 Tx, float2 Ty)
    {
        tq[32 * j] = make_float4(T.x, T.y, Tx.x, Tx.y);
        ty[32 * j] = Ty;
    }
    __device__ __forceinline__ void get(int j, float2& T, float2& Tx, float2& Ty) const
    {
        const float4 q = tq[32 * j];
        T = make_float2(q.x, q.y);
        Tx = make_float2(q.z, q.w);
        Ty = ty[32 * j];
    }
    float2* mk;  // cross-based support: 0/1 mask of slot j's two samples at mk[32 j]
    int off[SLP];
    float msk[SLP];
    int eo0[2], eo1[2];
    unsigned vbits;
    int roff[2];
    float rkeep[2];
    bool last_ok;
};

// First slot that can hold a vertical pair (SLP for the runtime layout).
template <int G, int SLP, int RC>
__host__ __device__ constexpr int first_generic_slot()
{
    if constexpr (RunLayout<G, RC>::on) return RunLayout<G, RC>::first_generic;
    return RC ? Layout<RC>::nh / G : SLP;
}

// Adds one pair's terms at its interpolated frame-2 values less the illumination
// offset, Jc = J - c (template of slot j; hci = (c - b)^-1 c of the Hampel weight,
// or 0 to give the pair weight 0).
template <int SLP, int MODEL, int RC, bool CROSS, int FG>
__device__ __forceinline__ void pair_terms(const Support<SLP>& S, float2 (&acc)[14], int j, float2 Jc, float2 ng1,
                                           float ha, float icb, float hci)
{
    float2 T, Tx, Ty;
    S.get(j, T, Tx, Ty);
    float2 r;
    if (MODEL == 4)
        r = __ffma2_rn(ng1, T, Jc);
    else
        r = __ffma2_rn(f2(-1.f), T, Jc);
    // only a generic slot (and any slot of the runtime layout) can hold a sample
    // past the support
    float2 w = make_float2(hampel_weight(r.x, ha, icb, hci), hampel_weight(r.y, ha, icb, hci));
    if (RC == 0 || j >= FG) w.y *= S.msk[j];
    if (CROSS) w = __fmul2_rn(w, S.mk[32 * j]);
    const float2 wTx = __fmul2_rn(w, Tx), wTy = __fmul2_rn(w, Ty);
    acc[0] = __ffma2_rn(wTx, Tx, acc[0]);
    acc[1] = __ffma2_rn(wTx, Ty, acc[1]);
    acc[4] = __ffma2_rn(wTy, Ty, acc[4]);
    acc[10] = __ffma2_rn(wTx, r, acc[10]);
    acc[11] = __ffma2_rn(wTy, r, acc[11]);
    if (MODEL == 4) {
        const float2 wT = __fmul2_rn(w, T);
        acc[2] = __ffma2_rn(wTx, T, acc[2]);
        acc[3] = __fadd2_rn(acc[3], wTx);
        acc[5] = __ffma2_rn(wTy, T, acc[5]);
        acc[6] = __fadd2_rn(acc[6], wTy);
        acc[7] = __ffma2_rn(wT, T, acc[7]);
        acc[8] = __fadd2_rn(acc[8], wT);
        acc[9] = __fadd2_rn(acc[9], w);
        acc[12] = __ffma2_rn(wT, r, acc[12]);
        acc[13] = __ffma2_rn(w, r, acc[13]);
    }
}

// The terms of run k of the run layout (N pairs from slot j0): each tap row is read
// once, as the bottom row of one pair and the top row of the next. The pairs that
// can be pads (all of a radius-5 run, the last of a radius-4 run) take the run's
// 0/1 weight factor.
template <typename TS, int SLP, int MODEL, int RC, bool CROSS, int FG, int N>
__device__ __forceinline__ void run_terms(const Support<SLP>& S, float2 (&acc)[14], const TapBlock<TS>& tb, int k,
                                          int j0, float2 ng1, float2 nc, float ha, float icb, float hc_icb)
{
    constexpr int first_pad = RC == 5 ? 0 : N - 1;  // first pair that can be a pad
    const float hci_pad = hc_icb * S.rkeep[k];
    const TS* pu = tb.base_u + S.roff[k];
    const TS* ps = tb.base_s + S.roff[k];
    typename TapBlock<TS>::Row top = tb.row(pu, ps, 0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const typename TapBlock<TS>::Row bot = tb.row(pu, ps, i + 1);
        pair_terms<SLP, MODEL, RC, CROSS, FG>(S, acc, j0 + i, tb.pair_rows(top, bot, nc), ng1, ha, icb,
                                              i >= first_pad ? hci_pad : hc_icb);
        top = bot;
    }
}

// Accumulates the weighted normal equations of the lane's pairs at one iterate.
// acc[0..9] = sum w (TxTx, TxTy, TxT, Tx, TyTy, TyT, Ty, TT, T, 1); acc[10..13] =
// sum w r (Tx, Ty, T, 1), each as .x/.y partial sums of a pair's two samples.
// Taps are read without clamping (TapBlock). In the run layout each run walks its
// len + 1 tap rows once, a row serving as the bottom of one pair and the top of
// the next.
template <typename TS, int G, int SLP, int MODEL, int RC, bool CROSS>
__device__ __forceinline__ void accumulate(const Support<SLP>& S, float2 (&acc)[14], const TapBlock<TS>& tb,
                                           const PairWeights& pw, int lane, int np, float g1, float c, float ha,
                                           float icb, float hc_icb)
{
    constexpr int FG = first_generic_slot<G, SLP, RC>();
    constexpr int J0 = RunLayout<G, RC>::on ? FG : 0;  // first slot of the loop below
    const float2 ng1 = f2(-g1), nc = f2(-c);
    if constexpr (RunLayout<G, RC>::on) {
        using RL = RunLayout<G, RC>;
        static_assert(RL::slots == SLP, "run layout slot count");
        if constexpr (RL::la == RL::lb) {
#pragma unroll
            for (int k = 0; k < 2; ++k)
                run_terms<TS, SLP, MODEL, RC, CROSS, FG, RL::la>(S, acc, tb, k, k * RL::la, ng1, nc, ha, icb, hc_icb);
        } else {
            run_terms<TS, SLP, MODEL, RC, CROSS, FG, RL::la>(S, acc, tb, 0, 0, ng1, nc, ha, icb, hc_icb);
            run_terms<TS, SLP, MODEL, RC, CROSS, FG, RL::lb>(S, acc, tb, 1, RL::la, ng1, nc, ha, icb, hc_icb);
        }
    }
#pragma unroll
    for (int j = J0; j < SLP; ++j) {
        // only the last slot can hold pairs past the support; testing it there
        // alone leaves the loads of all other slots free to be hoisted
        if (j == SLP - 1) {
            if (RunLayout<G, RC>::on ? !S.last_ok : lane + G * j >= np) break;
        }
        // the radius-4 run layout's generic slot holds vertical pairs only
        const bool vert = (RunLayout<G, RC>::on && RC == 4) || ((S.vbits >> (j - FG)) & 1u);
        const float2 Jc =
            j >= FG ? tb.generic(S.off[j], S.eo0[j - FG], S.eo1[j - FG], vert, pw, nc) : tb.pair(S.off[j], nc);
        pair_terms<SLP, MODEL, RC, CROSS, FG>(S, acc, j, Jc, ng1, ha, icb, hc_icb);
    }
}

// Writes one point's results (lane 0 of its group).
__device__ __forceinline__ void write_point(const dgf::TrackJob& J, int pt, int status, float fx, float fy,
                                            int iters, float m, float c, bool model4)
{
    const bool ok = status == DGF_TRACKED || status == DGF_MAXITER;
    reinterpret_cast<float2*>(J.flow)[pt] = ok ? make_float2(fx, fy) : make_float2(0.f, 0.f);
    J.status[pt] = (uint8_t)status;
    if (J.iters) J.iters[pt] = (uint8_t)min(iters, 255);
    if (J.illum) reinterpret_cast<float2*>(J.illum)[pt] = ok && model4 ? make_float2(m, c) : make_float2(0.f, 0.f);
}

// Job holding global point index gp (binary search over the prefix counts).
__device__ __forceinline__ int find_job(const TrackBatch& a, int gp)
{
    int job = 0;
    for (int lo = 0, hi = a.n_jobs - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (a.jobs[mid].pt_begin <= gp) {
            job = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    return job;
}

// Planes and size of level l of a job's pyramids.
template <typename TS>
struct LevelView {
    const TS *I1, *I1x, *I1y, *I2;
    int W, H, pitch;
    __device__ __forceinline__ LevelView(const dgf::TrackJob& J, int levels, int l)
    {
        dgf::LevelGeom g;
        dgf::level_geom(J.W, J.H, levels, (int)sizeof(TS), l, &g);
        I1 = reinterpret_cast<const TS*>(J.pyr1 + g.off_I);
        I1x = reinterpret_cast<const TS*>(J.pyr1 + g.off_Ix);
        I1y = reinterpret_cast<const TS*>(J.pyr1 + g.off_Iy);
        I2 = reinterpret_cast<const TS*>(J.pyr2 + g.off_I);
        W = g.W;
        H = g.H;
        pitch = g.pitch;
    }
};

// Level set-up: samples the template T, Tx, Ty at p_l + k into the lane's pairs
// and applies the minimum-eigenvalue test. Returns false for SMALL_EIG.
// Adaptive cross-based support of the level (CROSS): rows t = 0 .. 2R of the support
// (ky = t - R), one lane per row, scan their arms in frame 1's intensity plane around
// the centre pixel c (p_l rounded half up, clamped): arm[3t], arm[3t+1] = left and
// right arm lengths from the row's centre-column pixel a (at most R, while pixels
// differ from I(a) by at most tau), arm[3t+2] = |I(a) - I(c)| <= tau. The arms go to
// the group's rows of the per-warp reduction scratch (unused during the set-up); the
// vertical arm lengths up, dn follow from the row flags. Pixels are read clamped.
template <typename TS, int G>
__device__ __forceinline__ void cross_arms(const LevelView<TS>& L, float plx, float ply, int lane, unsigned mask,
                                           int R, float tau, int* arm, int& up, int& dn)
{
    const int cx = min(max((int)floorf(plx + 0.5f), 0), L.W - 1);
    const int cy = min(max((int)floorf(ply + 0.5f), 0), L.H - 1);
    const float vc = dgf::ld(L.I1 + (size_t)cy * L.pitch + cx);
    for (int t = lane; t < 2 * R + 1; t += G) {
        const TS* row = L.I1 + (size_t)min(max(cy + t - R, 0), L.H - 1) * L.pitch;
        const float va = dgf::ld(row + cx);
        int lf = 0, rt = 0;
        while (lf < R && fabsf(dgf::ld(row + max(cx - lf - 1, 0)) - va) <= tau) ++lf;
        while (rt < R && fabsf(dgf::ld(row + min(cx + rt + 1, L.W - 1)) - va) <= tau) ++rt;
        arm[3 * t] = lf;
        arm[3 * t + 1] = rt;
        arm[3 * t + 2] = fabsf(va - vc) <= tau;
    }
    __syncwarp(mask);
    up = 0;
    while (up < R && arm[3 * (R - up - 1) + 2]) ++up;
    dn = 0;
    while (dn < R && arm[3 * (R + dn + 1) + 2]) ++dn;
}

template <typename TS, int G, int SLP, int RC, bool CROSS>
__device__ __forceinline__ bool setup_level(Support<SLP>& S, const LevelView<TS>& L, float plx, float ply, int lane,
                                            unsigned mask, int R, float min_eig, float tau, WarpScratch& ws)
{
    constexpr int FG = first_generic_slot<G, SLP, RC>();
    const int side = 2 * R + 1;
    const float fx0 = floorf(plx), fy0 = floorf(ply);
    const int bx = (int)fx0 - R, by = (int)fy0 - R;
    const PairWeights pw(plx - fx0, ply - fy0);
    // the template's taps read without clamping when they lie within the planes'
    // replicated border, as they do for every point inside the frame (points given
    // outside it take the clamped reads)
    const bool direct = bx >= -dgf::kApron && bx + 2 * R + 2 <= L.W + dgf::kApron - 1 && by >= -dgf::kApron &&
                        by + 2 * R + 1 <= L.H + dgf::kApron - 1;
    const TapBlock<TS> tT(L.I1, L.pitch, bx, by, pw), tX(L.I1x, L.pitch, bx, by, pw), tY(L.I1y, L.pitch, bx, by, pw);
    float2 g00 = f2(0.f), g01 = f2(0.f), g11 = f2(0.f);
    float kept = 0.f;  // cross-based support: kept samples of the lane
    int* arm = nullptr;
    int up = 0, dn = 0;
    if (CROSS) {
        arm = reinterpret_cast<int*>(ws.rows + ((threadIdx.x & 31) - lane) * kRowStride);
        cross_arms<TS, G>(L, plx, ply, lane, mask, R, tau, arm, up, dn);
    }
    // mask of the sample at support coordinates (sx, sy), 0 .. 2R
    auto in_cross = [&](int sx, int sy) -> float {
        const int ky = sy - R, kx = sx - R;
        if (ky < -up || ky > dn) return 0.f;
        return kx >= -arm[3 * sy] && kx <= arm[3 * sy + 1] ? 1.f : 0.f;
    };
    S.vbits = 0u;
    S.last_ok = true;
#pragma unroll
    for (int j = 0; j < SLP; ++j) {
        float2 T = f2(0.f), Tx = f2(0.f), Ty = f2(0.f);
        float msk = 0.f;
        int off = 0;
        int x, y;  // tap origin of sample A in the support
        bool vert;
        const bool has = slot_origin<G, RC>(lane, j, R, x, y, vert);
        if (has) {
            off = y * L.pitch + x;
            msk = (vert ? y : x) + 1 < side ? 1.f : 0.f;
            // taps sample B adds in a generic slot: right column (horizontal), row
            // below (vertical), or, for the masked sample, two of A's own taps so
            // that every load stays inside the tap block
            const int e0 = vert ? (msk != 0.f ? off + 2 * L.pitch : off) : off + 2;
            const int e1 = vert ? e0 + 1 : off + L.pitch + 2;
            if (direct && j >= FG) {
                T = tT.generic(off, e0, e1, vert, pw);
                Tx = tX.generic(off, e0, e1, vert, pw);
                Ty = tY.generic(off, e0, e1, vert, pw);
            } else if (direct) {
                T = tT.pair(off);
                Tx = tX.pair(off);
                Ty = tY.pair(off);
            } else if (vert) {
                T = vpair_clamped(L.I1, L.pitch, L.W, L.H, bx + x, by + y, pw);
                Tx = vpair_clamped(L.I1x, L.pitch, L.W, L.H, bx + x, by + y, pw);
                Ty = vpair_clamped(L.I1y, L.pitch, L.W, L.H, bx + x, by + y, pw);
            } else {
                T = pair_clamped(L.I1, L.pitch, L.W, L.H, bx + x, by + y, pw);
                Tx = pair_clamped(L.I1x, L.pitch, L.W, L.H, bx + x, by + y, pw);
                Ty = pair_clamped(L.I1y, L.pitch, L.W, L.H, bx + x, by + y, pw);
            }
            if (msk == 0.f) T.y = Tx.y = Ty.y = 0.f;
            if (j >= FG) {
                S.eo0[j - FG] = e0;
                S.eo1[j - FG] = e1;
                if (vert) S.vbits |= 1u << (j - FG);
            }
        } else if (j >= FG) {
            S.eo0[j - FG] = S.eo1[j - FG] = 0;
        }
        if constexpr (RunLayout<G, RC>::on) {
            using RL = RunLayout<G, RC>;
            if (j == 0 || j == RL::la) S.roff[j == 0 ? 0 : 1] = off;  // a run's first tap row
            // the factor of the run's pads: all of a radius-5 run is a pad or none; the
            // last pair of a radius-4 run is one whenever any is
            if (j < FG && (RC == 5 ? j % RL::la == 0 : j == RL::la - 1 || j == FG - 1))
                S.rkeep[j < RL::la ? 0 : 1] = has ? 1.f : 0.f;
            if (j == SLP - 1) S.last_ok = has;
        }
        S.put(j, T, Tx, Ty);
        S.off[j] = off;
        S.msk[j] = msk;
        if (CROSS) {
            float2 mkv = f2(0.f);
            if (has) {
                mkv.x = in_cross(x, y);
                if (msk != 0.f) mkv.y = vert ? in_cross(x, y + 1) : in_cross(x + 1, y);
            }
            S.mk[32 * j] = mkv;
            kept += mkv.x + mkv.y;
            const float2 Txm = __fmul2_rn(Tx, mkv), Tym = __fmul2_rn(Ty, mkv);
            g00 = __ffma2_rn(Txm, Tx, g00);
            g01 = __ffma2_rn(Txm, Ty, g01);
            g11 = __ffma2_rn(Tym, Ty, g11);
        } else {
            g00 = __ffma2_rn(Tx, Tx, g00);
            g01 = __ffma2_rn(Tx, Ty, g01);
            g11 = __ffma2_rn(Ty, Ty, g11);
        }
    }
    const float G00 = group_sum<G>(g00.x + g00.y, mask);
    const float G01 = group_sum<G>(g01.x + g01.y, mask);
    const float G11 = group_sum<G>(g11.x + g11.y, mask);
    const float n_kept = CROSS ? group_sum<G>(kept, mask) : (float)(side * side);
    if (CROSS) __syncwarp(mask);  // every lane has read the arms before the scratch is reused
    const float ht = 0.5f * (G00 + G11), hd = 0.5f * (G00 - G11);
    const float lam = ht - sqrtf(hd * hd + G01 * G01);
    return !(lam / n_kept < min_eig);
}

// One Gauss-Newton step at iterate q (inside the level): accumulates, reduces and
// solves the weighted normal equations. Returns false on a non-positive pivot. The
// tap block of a position inside the level lies within the planes' replicated
// border (columns bx .. bx + 2R + 2, rows by .. by + 2R + 1), so no tap is clamped.
template <typename TS, int G, int SLP, int MODEL, int RC, bool CROSS>
__device__ __forceinline__ bool gn_step(const Support<SLP>& S, const LevelView<TS>& L, float qx, float qy, float m,
                                        float c, int lane, unsigned mask, int R, float ha, float icb, float hc_icb,
                                        WarpScratch& ws, float (&delta)[4])
{
    const int side = 2 * R + 1, pc = R + 1, np = RC ? Layout<RC>::np : side * pc;
    const float fx0 = floorf(qx), fy0 = floorf(qy);
    const int bx = (int)fx0 - R, by = (int)fy0 - R;
    const PairWeights pw(qx - fx0, qy - fy0);
    float2 acc[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) acc[k] = f2(0.f);
    const TapBlock<TS> tb(L.I2, L.pitch, bx, by, pw);
    accumulate<TS, G, SLP, MODEL, RC, CROSS>(S, acc, tb, pw, lane, np, 1.f + m, c, ha, icb, hc_icb);
    float h[16];
    if (MODEL == 4) {
        float v[16];
#pragma unroll
        for (int k = 0; k < 14; ++k) v[k] = acc[k].x + acc[k].y;
        v[14] = v[15] = 0.f;
        group_allreduce16<G>(v, h, mask, lane, ws);
        // a = (Tx, Ty, -T, -1): fold the signs of the T and constant columns
        float Hm[4][4] = {{h[0], h[1], -h[2], -h[3]},
                          {h[1], h[4], -h[5], -h[6]},
                          {-h[2], -h[5], h[7], h[8]},
                          {-h[3], -h[6], h[8], h[9]}};
        const float rhs[4] = {-h[10], -h[11], h[12], h[13]};
        return block_solve4(Hm, rhs, delta);
    }
    const float h0 = group_sum<G>(acc[0].x + acc[0].y, mask);
    const float h1 = group_sum<G>(acc[1].x + acc[1].y, mask);
    const float h4 = group_sum<G>(acc[4].x + acc[4].y, mask);
    const float b0 = group_sum<G>(acc[10].x + acc[10].y, mask);
    const float b1 = group_sum<G>(acc[11].x + acc[11].y, mask);
    float Hm[2][2] = {{h0, h1}, {h1, h4}};
    const float rhs[2] = {-b0, -b1};
    float x[2];
    const bool ok = chol_solve<2>(Hm, rhs, x);
    delta[0] = x[0];
    delta[1] = x[1];
    delta[2] = delta[3] = 0.f;
    return ok;
}

// One point per group, coarse-to-fine loops kept tight. Blocks are short-lived
// (eight points each at 16 lanes), so the block scheduler balances points of
// uneven iteration counts and pairs of uneven size; a persistent variant that
// pulled points from a work counter through a per-group state machine measured
// slower on both the single-pair and the 64-pair workloads.
template <typename TS, int G, int SLP, int MODEL, int MINB, int RC, bool CROSS>
__global__ void __launch_bounds__(block_threads<G>(), MINB) rlof_kernel(const __grid_constant__ TrackBatch a)
{
    const int gp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (gp >= a.total) return;
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int R = RC ? RC : a.radius;
    const float icb = a.inv_cb, hc_icb = a.hc * a.inv_cb;
    const dgf::TrackJob& J = a.jobs[find_job(a, gp)];
    const int pt = gp - J.pt_begin;
    if (J.gate) {  // gated out: the whole group leaves (the kernel has no block barrier)
        const uint8_t gs = J.gate[pt];
        if (gs != DGF_TRACKED && gs != DGF_MAXITER) {
            if (lane == 0) write_point(J, pt, gs, 0.f, 0.f, 0, 0.f, 0.f, MODEL == 4);
            return;
        }
    }
    constexpr int NW = block_threads<G>() / 32;  // warps per block
    __shared__ WarpScratch s_ws[NW];
    WarpScratch& ws = s_ws[threadIdx.x >> 5];
    Support<SLP> S;
    __shared__ float4 s_tq[NW][SLP][32];
    __shared__ float2 s_ty[NW][SLP][32];
    S.tq = &s_tq[threadIdx.x >> 5][0][threadIdx.x & 31];
    S.ty = &s_ty[threadIdx.x >> 5][0][threadIdx.x & 31];
    __shared__ float2 s_mk[CROSS ? NW : 1][CROSS ? SLP : 1][32];
    S.mk = CROSS ? &s_mk[threadIdx.x >> 5][0][threadIdx.x & 31] : nullptr;

    const float2 p = reinterpret_cast<const float2*>(J.pts)[(long long)pt * J.pt_stride];
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f, m = 0.f, c = 0.f;
    if (J.prior) {
        // global-motion prior: level-0 flow A p + t - p, scaled to the coarsest level
        const double* q = J.prior;
        const double x = p.x, y = p.y, s0 = ldexp(1.0, -(a.levels - 1));
        gx = (float)((q[0] * x + q[1] * y + q[2] - x) * s0);
        gy = (float)((q[3] * x + q[4] * y + q[5] - y) * s0);
    }
    int status = DGF_TRACKED, iters = 0;

    for (int l = a.levels - 1; l >= 0; --l) {
        const LevelView<TS> L(J, a.pyr_levels, l);
        const float scale = __int_as_float((127 - l) << 23);  // 2^-l
        const float plx = (p.x + 0.5f) * scale - 0.5f, ply = (p.y + 0.5f) * scale - 0.5f;
        if (!setup_level<TS, G, SLP, RC, CROSS>(S, L, plx, ply, lane, mask, R, a.min_eig, a.cross_tau, ws)) {
            status = DGF_SMALL_EIG;
            break;
        }
        dx = 0.f;
        dy = 0.f;
        bool converged = false;
        for (int it = 0; it < a.max_iter; ++it) {
            const float qx = plx + gx + dx, qy = ply + gy + dy;
            if (!(qx >= 0.f && qx <= (float)(L.W - 1) && qy >= 0.f && qy <= (float)(L.H - 1))) {
                status = DGF_OOB;
                break;
            }
            float delta[4];
            if (!gn_step<TS, G, SLP, MODEL, RC, CROSS>(S, L, qx, qy, m, c, lane, mask, R, a.ha, icb, hc_icb, ws,
                                                       delta)) {
                status = DGF_SINGULAR;
                break;
            }
            dx += delta[0];
            dy += delta[1];
            if (MODEL == 4) {
                m += delta[2];
                c += delta[3];
            }
            ++iters;
            if (delta[0] * delta[0] + delta[1] * delta[1] < a.eps2) {
                converged = true;
                break;
            }
        }
        if (status != DGF_TRACKED) break;
        if (l > 0) {
            gx = 2.f * (gx + dx);
            gy = 2.f * (gy + dy);
        } else if (!converged) {
            status = DGF_MAXITER;
        }
    }
    if (lane == 0) write_point(J, pt, status, gx + dx, gy + dy, iters, m, c, MODEL == 4);
}

// Set by dgf_rlof_set_lanes from any thread, read when a launch is configured.
std::atomic<int> g_lanes_override{0};

template <typename TS, int MODEL, int G, int SLP, int RC>
int launch_one(const TrackBatch& a, cudaStream_t stream)
{
    const long long total = (long long)a.total * G;
    constexpr int BT = block_threads<G>();
    const unsigned grid = (unsigned)((total + BT - 1) / BT);
    if (a.cross_tau > 0.f)
        rlof_kernel<TS, G, SLP, MODEL, min_blocks<G, RC, true>(), RC, true><<<grid, BT, 0, stream>>>(a);
    else
        rlof_kernel<TS, G, SLP, MODEL, min_blocks<G, RC, false>(), RC, false><<<grid, BT, 0, stream>>>(a);
    return dgf::launch_status();
}

template <typename TS, int MODEL>
int launch(const TrackBatch& a, int lanes, cudaStream_t stream)
{
    // radius 4 and 5: compile-time layout with the vertical last column
#define DGF_LAUNCH_RC(G, RC) \
    if (lanes == G && a.radius == RC) return launch_one<TS, MODEL, G, (Layout<RC>::np + G - 1) / G, RC>(a, stream);
    DGF_LAUNCH_RC(8, 4)
    DGF_LAUNCH_RC(8, 5)
    DGF_LAUNCH_RC(16, 4)
    DGF_LAUNCH_RC(16, 5)
    DGF_LAUNCH_RC(32, 4)
    DGF_LAUNCH_RC(32, 5)
#undef DGF_LAUNCH_RC
    // other radii: runtime layout, 32 lanes
    const int np = (2 * a.radius + 1) * (a.radius + 1);  // sample pairs in the support
#define DGF_LAUNCH(G, SLP) \
    if (lanes == G && (np + G - 1) / G == SLP) return launch_one<TS, MODEL, G, SLP, 0>(a, stream);
    DGF_LAUNCH(32, 1)   // radius 1..3
    DGF_LAUNCH(32, 3)   // radius 6
    DGF_LAUNCH(32, 4)   // radius 7
#undef DGF_LAUNCH
    return DGF_ERR_ARG;
}

int choose_lanes(int radius, int set)
{
    // 8 and 16 lanes are built for radius 4 and 5 only; other radii use 32 lanes.
    // Measured on GB300: both radii fastest at 8 lanes (radius 5 on the 1242x375 pair:
    // 1.25 ms against 1.40 ms at 16 lanes, once no two points of a warp take
    // different tap-load paths; radius 4 on its step-4 pair: 0.224 against 0.226 ms).
    // The choice does not depend on the launch's size, so a pair gives the same bits
    // alone and inside a batch (16 lanes would shorten launches of at most 16 points a
    // SM, the 256x128 pair's 1,953 points 0.088 against 0.096 ms, not taken for that).
    if (radius != 4 && radius != 5) return 32;
    if (set) return set;
    return 8;
}

}  // namespace rlof_detail

using namespace rlof_detail;

extern "C" void dgf_rlof_params_default(dgf_rlof_params* p)
{
    if (!p) return;
    p->version = DGF_RLOF_PARAMS_VERSION;
    p->levels = 3;
    p->radius = 4;
    p->max_iter = 30;
    p->model = 4;
    p->storage = DGF_F32;
    p->eps = 1e-3f;
    p->hampel_a = 8.f;
    p->hampel_b = 16.f;
    p->hampel_c = 32.f;
    p->min_eig = 1e-3f;
    p->cross_tau = 0.f;
}

// Tuning hook: lanes per point (8, 16 or 32; 0 restores the automatic choice).
// Returns the previous setting, or DGF_ERR_ARG for an unsupported value.
extern "C" int dgf_rlof_set_lanes(int lanes)
{
    if (lanes != 0 && lanes != 8 && lanes != 16 && lanes != 32) return DGF_ERR_ARG;
    return g_lanes_override.exchange(lanes, std::memory_order_relaxed);
}

namespace dgf {

// Validates tracking parameters; fills the shared fields of a launch.
int prepare_params(const dgf_rlof_params* p, TrackBatch& a)
{
    if (!p || p->version != DGF_RLOF_PARAMS_VERSION) return DGF_ERR_ARG;
    if (p->levels < 1 || p->levels > DGF_MAX_LEVELS || p->radius < 1 || p->radius > DGF_MAX_RADIUS ||
        p->max_iter < 1 || p->max_iter > 255 || (p->model != 2 && p->model != 4) ||
        (p->storage != DGF_F32 && p->storage != DGF_F16) || !(p->eps >= 0.f) || !(p->hampel_a > 0.f) ||
        !(p->hampel_b >= p->hampel_a) || !(p->hampel_c > p->hampel_b) || !(p->min_eig >= 0.f) ||
        !(p->cross_tau >= 0.f))
        return DGF_ERR_ARG;
    a.levels = p->levels;
    a.pyr_levels = p->levels;
    a.radius = p->radius;
    a.max_iter = p->max_iter;
    a.es = p->storage == DGF_F32 ? 4 : 2;
    a.eps2 = p->eps * p->eps;
    a.ha = p->hampel_a;
    a.hc = p->hampel_c;
    a.inv_cb = 1.f / (p->hampel_c - p->hampel_b);
    a.min_eig = p->min_eig;
    a.cross_tau = p->cross_tau;
    return DGF_OK;
}

// Coarsest level large enough for the support (2 radius + 2 taps).
int check_levels(int W, int H, const dgf_rlof_params* p)
{
    dgf::LevelGeom g;
    if (!dgf::level_geom(W, H, p->levels, p->storage == DGF_F32 ? 4 : 2, p->levels - 1, &g)) return DGF_ERR_ARG;
    const int need = 2 * p->radius + 2;
    return g.W < need || g.H < need ? DGF_ERR_LEVELS : DGF_OK;
}

int lanes_setting() { return ::rlof_detail::g_lanes_override.load(std::memory_order_relaxed); }

int launch_track(const TrackBatch& a, const dgf_rlof_params* p, cudaStream_t stream, int lanes_set)
{
    using namespace ::rlof_detail;
    const int lanes = choose_lanes(p->radius, lanes_set >= 0 ? lanes_set : lanes_setting());
    if (p->storage == DGF_F32)
        return p->model == 4 ? launch<float, 4>(a, lanes, stream) : launch<float, 2>(a, lanes, stream);
    return p->model == 4 ? launch<__half, 4>(a, lanes, stream) : launch<__half, 2>(a, lanes, stream);
}

}  // namespace

extern "C" int rlof_track(const void* pyr1, const void* pyr2, int W, int H, const float* pts, int n,
                          const dgf_rlof_params* p, float* flow, uint8_t* status, uint8_t* iters, float* illum,
                          cudaStream_t stream)
{
    TrackBatch a = {};
    int rc = dgf::prepare_params(p, a);
    if (rc == DGF_OK) rc = n < 0 || W < 1 || H < 1 ? DGF_ERR_ARG : dgf::check_levels(W, H, p);
    if (rc != DGF_OK) return rc;
    if (n == 0) return DGF_OK;
    if (!pyr1 || !pyr2 || !pts || !flow || !status || !dgf::aligned(pyr1, 256) || !dgf::aligned(pyr2, 256) ||
        !dgf::aligned(pts, 8) || !dgf::aligned(flow, 8) || (illum && !dgf::aligned(illum, 8)))
        return DGF_ERR_ARG;
    a.n_jobs = 1;
    a.total = n;
    a.jobs[0] = dgf::TrackJob{static_cast<const char*>(pyr1), static_cast<const char*>(pyr2), W, H, pts, flow, status,
                              iters, illum, 0, 1, nullptr};
    return dgf::launch_track(a, p, stream);
}
