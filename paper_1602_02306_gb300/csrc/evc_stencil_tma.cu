// evc_stencil_tma.cu -- the stencil pass of evc_stencil.cu (the same
// operator, operands and arithmetic, point by point: the passes of
// C = M (H - sigma I) M and of the Chebyshev factors of M, Sec. 2 Eq. negi_T
// and Sec. 6) with block tiles staged by the tensor memory accelerator.
//
// A block owns a TX x TY tile of (x, y) points of one chunk and marches it
// along z.  For every plane it loads, with tiled tensor copies
// (cp.async.bulk.tensor) into shared memory: the tile's points of the input
// vector and the R-wide arms of the stencil around the tile (x arms TY x R,
// y arms R x TX; periodic wrap by the arms' start coordinates), and the tile
// of each pointwise operand.  One elected lane per box issues the copy; an
// mbarrier per ring stage counts the bytes.  Each thread computes a 2 x 2
// patch of points and 16-byte column vectors of them (as the patch kernel
// does): z neighbours come from a register window, in-patch neighbours from
// registers, the others from the shared tile, so every input vector of a
// plane is read from L2 once per block instead of once per thread that
// needs it, and no loaded byte passes through L1.
//
// Two rings, filled by a producer warp while four consumer warps compute:
// stage A (the input's tile and arms) runs R + 1 planes or more ahead of the
// plane computed -- the register window takes plane z + R + 1 from it when
// plane z is done -- and stage B (pointwise operands) one plane behind stage
// A.  A stage is refilled once every consumer warp has released the plane it
// held.  Every wait is bounded and records DERR_TIMEOUT; a block waits for
// its own copies in flight before it exits.
#include "evc_internal.cuh"
#include "evc_bulk.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <mutex>

namespace evc {
namespace {

template <typename T> struct alignas(16) Pack { T v[16 / sizeof(T)]; };
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; };
template <> struct Vec16<double> { typedef double2 type; };

template <typename T>
__device__ __forceinline__ Pack<T> ldg_pack(const Pack<T>* p)
{
    typename Vec16<T>::type t = __ldg(reinterpret_cast<const typename Vec16<T>::type*>(p));
    Pack<T> r;
    memcpy(&r, &t, 16);
    return r;
}

template <typename T>
__device__ __forceinline__ void st_pack(Pack<T>* p, const Pack<T>& v)
{
    typename Vec16<T>::type t;
    memcpy(&t, &v, 16);
    *reinterpret_cast<typename Vec16<T>::type*>(p) = t;
}

enum { HAS_X = 1, HAS_PREV = 2, HAS_PP = 4, HAS_VS = 8 };   // as in evc_stencil.cu

struct TmaArgs {
    StencilPass p;
    StencilOp op;
    const int* shift_of;
    const double* sigma;
    const void* jac;
    const int* chunk_active;
    int64_t n;
    int* err;
};

// Tensor maps of one pass, each over [chunk][z][y][x][CW] of one operand:
// the input's interior box (CW, TX, TY), x-arm box (CW, R, TY) and y-arm box
// (CW, TX, R); the interior boxes of the pointwise operands present.
struct TmaMaps {
    CUtensorMap in_c, in_x, in_y;
    CUtensorMap op[3];
};

constexpr int kTmaThreads = 128;
constexpr int TMX = 8;                                    // tile points along x
template <typename T>
__host__ __device__ constexpr int tma_ty() { return sizeof(T) == 4 ? 8 : 4; }   // along y

template <int MASK>
__host__ __device__ constexpr int tma_nop()
{
    return ((MASK & HAS_X) ? 1 : 0) + ((MASK & HAS_PREV) ? 1 : 0) + ((MASK & HAS_PP) ? 1 : 0);
}
// Points of one stage: A = the input's tile and the stencil arms around it
// (x arms TY x R on both sides, y arms R x TX below and above); B = the tiles
// of the pointwise operands.
template <typename T, int R>
__host__ __device__ constexpr int tma_a_pts() { return TMX * tma_ty<T>() + 2 * tma_ty<T>() * R + 2 * R * TMX; }
template <typename T, int MASK>
__host__ __device__ constexpr int tma_b_pts() { return tma_nop<MASK>() * TMX * tma_ty<T>(); }
template <typename T, int R, int MASK>
__host__ __device__ constexpr int tma_ring_bytes(int la, int lb)
{
    return (la * tma_a_pts<T, R>() + lb * tma_b_pts<T, MASK>()) * CW * (int)sizeof(T);
}

// Ring depths (LA, LB): the first of (R+3, 3), (R+3, 2), (R+2, 2) whose shared
// memory lets two blocks share an SM (111 KB each), else the first that fits
// one block.  Stage A runs LA - 1 planes ahead of the plane computed, the
// window's plane z + R + 1 LA - R - 2 planes ahead of its use.
template <typename T, int R, int MASK>
__host__ __device__ constexpr int tma_depth_code()
{
    constexpr int two = 111 * 1024, one = 220 * 1024;
    return tma_ring_bytes<T, R, MASK>(R + 3, 3) <= two   ? 0
           : tma_ring_bytes<T, R, MASK>(R + 3, 2) <= two ? 1
           : tma_ring_bytes<T, R, MASK>(R + 2, 2) <= two ? 2
           : tma_ring_bytes<T, R, MASK>(R + 3, 3) <= one ? 0
           : tma_ring_bytes<T, R, MASK>(R + 3, 2) <= one ? 1
                                                         : 2;
}
template <typename T, int R, int MASK>
__host__ __device__ constexpr int tma_la() { return tma_depth_code<T, R, MASK>() == 2 ? R + 2 : R + 3; }
template <typename T, int R, int MASK>
__host__ __device__ constexpr int tma_lb() { return tma_depth_code<T, R, MASK>() == 0 ? 3 : 2; }

// 5-d tiled tensor copy global -> shared, completion counted on bar in bytes.
__device__ __forceinline__ void tma_load5(void* dst, const CUtensorMap* map, int c1, int c2,
                                          int c3, int c4, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(smem_addr(bar))
        : "memory");
}

// Input planes z0 + t of a segment of nz planes that a block reads: the
// segment's own planes (in-plane neighbours) and, for the register window,
// planes z0 + R + 1 .. z0 + nz - 1 + R.  All of 0 .. nz + R - 1 unless the
// segment is R planes or shorter.
__device__ __forceinline__ bool tma_plane_needed(int t, int nz, int R)
{
    return t < nz || (t >= R + 1 && t < nz + R);
}

// Bounded wait for the phase of the given parity that also gives up once the
// block's failure flag is set; a wait that runs out sets the flag.
__device__ __forceinline__ bool mbar_wait_or(uint64_t* bar, uint32_t parity, volatile int* fail)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*fail) return false;
        if (clock64() - t0 > kWaitCycles) {
            *fail = 1;
            return false;
        }
    }
    return true;
}

// The same wait by every lane of a warp (each lane observes the phase, so the
// copied bytes are visible to it), with one outcome for the warp.
__device__ __forceinline__ bool mbar_wait_warp_or(uint64_t* bar, uint32_t parity, volatile int* fail)
{
    return __all_sync(0xffffffffu, mbar_wait_or(bar, parity, fail));
}

template <typename T, int R, int MASK, int PM>
__global__ void __launch_bounds__(kTmaThreads + 32)
stencil_tma_kernel(const __grid_constant__ TmaMaps maps, const TmaArgs a)
{
    static_assert(PM == PM_NONE || PM == PM_TLEFT, "the tiled pass scales no operand");
    constexpr bool ROWS = PM == PM_TLEFT;
    constexpr int W = 16 / sizeof(T);
    constexpr int LPP = CW / W;                  // threads per point
    constexpr int TX = TMX, TY = tma_ty<T>();
    constexpr int TXP = TX / 2;                  // 2 x 2 patches per tile row
    static_assert(TXP * (TY / 2) * LPP == kTmaThreads, "one patch per consumer thread");
    constexpr int NCW = kTmaThreads / 32;        // consumer warps; warp NCW issues the copies
    constexpr int NPT = 4;
    constexpr bool X = MASK & HAS_X, PREV = MASK & HAS_PREV, PP = MASK & HAS_PP,
                   VS = MASK & HAS_VS;
    constexpr int NOP = tma_nop<MASK>();
    constexpr int LA = tma_la<T, R, MASK>(), LB = tma_lb<T, R, MASK>();
    static_assert(LA >= R + 2 && (NOP == 0 || LB >= R), "the rings must not hold back the window's planes");
    constexpr int A_PTS = tma_a_pts<T, R>(), B_PTS = tma_b_pts<T, MASK>();
    // stage A layout, in points: the tile [TY][TX], x arms [TY][R] left and
    // right, y arms [R][TX] below and above (each the box's own order)
    constexpr int A_XL = TX * TY, A_XR = A_XL + TY * R, A_YB = A_XR + TY * R, A_YT = A_YB + R * TX;
    constexpr uint32_t PT_BYTES = CW * sizeof(T);
    constexpr uint32_t A_BYTES = A_PTS * PT_BYTES, B_BYTES = B_PTS * PT_BYTES;
    constexpr int NBX = 4 * R, NB = 8 * R;       // halo points of a 2 x 2 patch

    const int ch = blockIdx.z;
    if (!a.chunk_active[ch]) return;
    extern __shared__ __align__(128) unsigned char st_raw[];
    // tensor copies land on 128-byte boundaries (every stage and box is a
    // whole number of 128-byte points from the base)
    if (smem_addr(st_raw) & 127) {
        if (threadIdx.x == 0) atomicExch(a.err, DERR_BOUNDS);
        return;
    }
    Pack<T>* ringA = reinterpret_cast<Pack<T>*>(st_raw);            // [LA][A_PTS][LPP]
    Pack<T>* ringB = ringA + (size_t)LA * A_PTS * LPP;              // [LB][B_PTS][LPP]
    // full: the stage's bytes have landed; empty: every consumer warp is done
    // with the plane it held
    __shared__ uint64_t fullA[LA], fullB[LB], emptyA[LA], emptyB[LB];
    __shared__ int s_fail, s_lastA, s_lastB;
    __shared__ Pack<T> s_sig[LPP], s_insc[LPP], s_a0s[LPP], s_ppc[LPP];
    __shared__ int s_shift[CW];
    if (threadIdx.x < CW) {
        const int c = ch * CW + threadIdx.x;
        const int l = threadIdx.x / W, w = threadIdx.x % W;
        s_sig[l].v[w] = VS ? (T)a.sigma[c] : (T)0;
        s_insc[l].v[w] = a.p.insc ? (T)a.p.insc[c] : (T)1;
        s_a0s[l].v[w] = (T)(a.p.a0 * (a.p.xs ? a.p.xs[c] : 1.0));
        s_ppc[l].v[w] = PP ? (T)a.p.ppc[c] : (T)0;
        s_shift[threadIdx.x] = ROWS ? a.shift_of[c] : 0;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < LA; ++s) {
            mbar_init(&fullA[s], 1);
            mbar_init(&emptyA[s], NCW);
        }
        for (int s = 0; s < LB; ++s) {
            mbar_init(&fullB[s], 1);
            mbar_init(&emptyB[s], NCW);
        }
        s_fail = 0;
        s_lastA = -1;
        s_lastB = -1;
        mbar_init_fence();
    }
    __syncthreads();

    const int N = a.op.N;                        // a multiple of TX and TY (host check)
    const int warp = threadIdx.x >> 5, l32 = threadIdx.x & 31;
    const int tilesX = N / TX;
    const int x0 = (blockIdx.x % tilesX) * TX, y0 = (blockIdx.x / tilesX) * TY;
    const int zb = a.op.zb > 0 ? a.op.zb : 32;
    const int z0 = blockIdx.y * zb;
    const int z1 = min(z0 + zb, N);
    const int nz = z1 - z0;
    const int nA = nz + R;                       // planes z0 .. z1 - 1 + R of the input
    volatile int* fail = &s_fail;

    if (warp == NCW) {
        // Producer warp.  Step t issues the input's plane t (stage A: the tile
        // and its arms) and then the operands of plane t - 1 (stage B).
        // Consumers need A[p] and B[p] for plane p and A[p + R + 1] for their
        // register window; a stage is refilled once the plane it held is
        // released, so A[p + R + 1] waits on the release of planes
        // p + R + 1 - LA (A) and p + R - 1 - LB (B), both at most p - 1.
        const int xl = x0 == 0 ? N - R : x0 - R, xr = x0 + TX == N ? 0 : x0 + TX;
        const int yb = y0 == 0 ? N - R : y0 - R, yt = y0 + TY == N ? 0 : y0 + TY;
        for (int t = 0; t < nA + 1; ++t) {
            if (t < nA && tma_plane_needed(t, nz, R)) {
                const int s = t % LA, k = t / LA;
                bool ok = true;
                if (l32 == 0) {
                    if (k > 0) ok = mbar_wait_or(&emptyA[s], (k - 1) & 1, fail);
                    if (ok) {
                        mbar_arrive_expect_tx(&fullA[s], A_BYTES);
                        s_lastA = t;
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                const int zz = (z0 + t) % N;
                Pack<T>* b = ringA + (size_t)s * A_PTS * LPP;
                if (l32 == 0) tma_load5(b, &maps.in_c, x0, y0, zz, ch, &fullA[s]);
                else if (l32 == 1) tma_load5(b + A_XL * LPP, &maps.in_x, xl, y0, zz, ch, &fullA[s]);
                else if (l32 == 2) tma_load5(b + A_XR * LPP, &maps.in_x, xr, y0, zz, ch, &fullA[s]);
                else if (l32 == 3) tma_load5(b + A_YB * LPP, &maps.in_y, x0, yb, zz, ch, &fullA[s]);
                else if (l32 == 4) tma_load5(b + A_YT * LPP, &maps.in_y, x0, yt, zz, ch, &fullA[s]);
            }
            const int tb = t - 1;
            if (NOP > 0 && tb >= 0 && tb < nz) {
                const int s = tb % LB, k = tb / LB;
                bool ok = true;
                if (l32 == 0) {
                    if (k > 0) ok = mbar_wait_or(&emptyB[s], (k - 1) & 1, fail);
                    if (ok) {
                        mbar_arrive_expect_tx(&fullB[s], B_BYTES);
                        s_lastB = tb;
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                Pack<T>* b = ringB + (size_t)s * B_PTS * LPP;
                if (l32 < NOP) tma_load5(b + l32 * TX * TY * LPP, &maps.op[l32], x0, y0, z0 + tb, ch, &fullB[s]);
            }
        }
    } else {
        const int lane = threadIdx.x % LPP;
        const int pt = threadIdx.x / LPP;
        const int px = (pt % TXP) * 2, py = (pt / TXP) * 2;
        const int x = x0 + px, y = y0 + py;
        const int64_t NN = (int64_t)N * N;
        const int64_t n = a.n;
        const T* __restrict__ jac = static_cast<const T*>(a.jac);
        const T* __restrict__ V = static_cast<const T*>(a.op.V);
        const Pack<T>* in = reinterpret_cast<const Pack<T>*>(
            static_cast<const T*>(a.p.in) + ch * a.p.in_cs) + lane;
        Pack<T>* out = reinterpret_cast<Pack<T>*>(static_cast<T*>(a.p.out) + ch * a.p.out_cs) + lane;

        // stage-A point index of the halo points of the patch, in the order
        // of the patch kernel: per row b, x offsets -R..-1 and 2..R+1; per
        // column q, y offsets the same
        int hidx[NB];
        auto tile_index = [&](int tx, int ty) {
            return tx < 0     ? A_XL + ty * R + (tx + R)
                   : tx >= TX ? A_XR + ty * R + (tx - TX)
                   : ty < 0   ? A_YB + (ty + R) * TX + tx
                   : ty >= TY ? A_YT + (ty - TY) * TX + tx
                              : ty * TX + tx;
        };
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int d = 0; d < 2 * R; ++d)
                hidx[b * 2 * R + d] = tile_index(px + (d < R ? d - R : 2 + d - R), py + b);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int d = 0; d < 2 * R; ++d)
                hidx[NBX + q * 2 * R + d] = tile_index(px + q, py + (d < R ? d - R : 2 + d - R));

        int64_t cxy[NPT];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 2; ++q) cxy[b * 2 + q] = (x + q) + (int64_t)N * (y + b);

        // register window: planes z - R .. z + R of the patch's points
        Pack<T> win[2 * R + 1][NPT];
#pragma unroll
        for (int o = -R; o <= R; ++o) {
            const int64_t zq = NN * (((z0 + o) % N + N) % N);
#pragma unroll
            for (int q = 0; q < NPT; ++q) win[o + R][q] = ldg_pack(in + (cxy[q] + zq) * LPP);
        }

        const T k1 = (T)a.p.k1;
        const T c1 = (T)a.op.c1, c2 = (T)a.op.c2;
        const T dg = (T)(a.p.k1 * a.op.cd + a.p.k0);
        const T a2 = (T)a.p.a2;
        const Pack<T> sig = s_sig[lane], insc = s_insc[lane], a0c = s_a0s[lane], ppcc = s_ppc[lane];

        for (int it = 0; it < nz; ++it) {
            const int sa = it % LA, sb = NOP > 0 ? it % LB : 0;
            bool ok = mbar_wait_warp_or(&fullA[sa], (it / LA) & 1, fail);
            if (NOP > 0 && ok) ok = mbar_wait_warp_or(&fullB[sb], (it / LB) & 1, fail);
            if (!ok) break;
            const Pack<T>* stA = ringA + (size_t)sa * A_PTS * LPP + lane;
            const Pack<T>* stB = ringB + (size_t)sb * B_PTS * LPP + lane;
            const int z = z0 + it;
            const int64_t rowz = NN * z;
            auto halo = [&](int u) -> Pack<T> { return stA[hidx[u] * LPP]; };
#pragma unroll
            for (int b = 0; b < 2; ++b) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int pp_ = b * 2 + q;
                    // value of the plane-z point at offset (ox, oy) from point (q, b)
                    auto nbv = [&](int ox, int oy) -> Pack<T> {
                        const int xx = q + ox, yy = b + oy;
                        if (oy == 0) {
                            if (xx >= 0 && xx < 2) return win[R][b * 2 + xx];
                            return halo(b * 2 * R + (xx < 0 ? xx + R : R + xx - 2));
                        }
                        if (yy >= 0 && yy < 2) return win[R][yy * 2 + q];
                        return halo(NBX + q * 2 * R + (yy < 0 ? yy + R : R + yy - 2));
                    };
                    const Pack<T> xm1 = nbv(-1, 0), xp1 = nbv(1, 0), ym1 = nbv(0, -1), yp1 = nbv(0, 1);
                    Pack<T> xm2, xp2, ym2, yp2;
                    if (R == 2) {
                        xm2 = nbv(-2, 0);
                        xp2 = nbv(2, 0);
                        ym2 = nbv(0, -2);
                        yp2 = nbv(0, 2);
                    }
                    const T vp = VS ? __ldg(V + cxy[pp_] + rowz) : (T)0;
                    Pack<T> res;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        T off = c1 * (xm1.v[w] + xp1.v[w] + ym1.v[w] +
                                      yp1.v[w] + win[R - 1][pp_].v[w] + win[R + 1][pp_].v[w]);
                        if (R == 2)
                            off += c2 * (xm2.v[w] + xp2.v[w] + ym2.v[w] +
                                         yp2.v[w] + win[0][pp_].v[w] + win[2 * R][pp_].v[w]);
                        T stv = k1 * off + (dg + vp - sig.v[w]) * win[R][pp_].v[w];
                        if (ROWS)
                            stv *= __ldg(jac + (int64_t)s_shift[lane * W + w] * n + cxy[pp_] + rowz);
                        res.v[w] = insc.v[w] * stv;
                    }
                    const Pack<T>* opt = stB + ((py + b) * TX + (px + q)) * LPP;   // this point
                    int k = 0;
                    if (X) {
                        const Pack<T> t = opt[(k++) * TX * TY * LPP];
#pragma unroll
                        for (int w = 0; w < W; ++w) res.v[w] += a0c.v[w] * t.v[w];
                    }
                    if (PREV) {
                        const Pack<T> t = opt[(k++) * TX * TY * LPP];
#pragma unroll
                        for (int w = 0; w < W; ++w) res.v[w] -= a2 * t.v[w];
                    }
                    if (PP) {
                        const Pack<T> t = opt[(k++) * TX * TY * LPP];
#pragma unroll
                        for (int w = 0; w < W; ++w) res.v[w] -= ppcc.v[w] * t.v[w];
                    }
                    st_pack(out + (cxy[pp_] + rowz) * LPP, res);
                }
            }
            // plane it is done with: release its stages
            __syncwarp();
            if (l32 == 0) {
                mbar_arrive(&emptyA[sa]);
                if (NOP > 0) mbar_arrive(&emptyB[sb]);
            }
            if (it + 1 < nz) {
                // plane z + R + 1 enters the window
                const int ia = it + R + 1;
                if (!mbar_wait_warp_or(&fullA[ia % LA], (ia / LA) & 1, fail)) break;
                const Pack<T>* nx = ringA + (size_t)(ia % LA) * A_PTS * LPP + lane;
#pragma unroll
                for (int q = 0; q < NPT; ++q) {
                    const Pack<T> v = nx[((py + q / 2) * TX + (px + q % 2)) * LPP];
#pragma unroll
                    for (int o = 0; o < 2 * R; ++o) win[o][q] = win[o + 1][q];
                    win[2 * R][q] = v;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // every copy this block issued has landed before its shared memory is
        // released (after a failure some were never waited for); a wait that
        // ran out is recorded
        if (*fail) atomicCAS(a.err, DERR_NONE, DERR_TIMEOUT);
        for (int t = max(0, s_lastA - LA + 1); t <= s_lastA; ++t)
            if (tma_plane_needed(t, nz, R)) mbar_wait(&fullA[t % LA], (t / LA) & 1);
        for (int t = max(0, s_lastB - LB + 1); t <= s_lastB; ++t)
            mbar_wait(&fullB[t % LB], (t / LB) & 1);
    }
    __syncthreads();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// A map of one operand (base = its chunk c0, chunk stride cs elements) with
// box (CW, bx, by, 1, 1).
template <typename T>
bool encode_box(CUtensorMap* m, const void* base, int64_t cs, int N, int cn, int bx, int by)
{
    auto fn = encode_tiled();
    if (!fn || !base) return false;
    const cuuint64_t e = sizeof(T);
    const cuuint64_t vol = (cuuint64_t)CW * N * N * N;
    cuuint64_t dim[5] = {(cuuint64_t)CW, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)cn};
    cuuint64_t str[4] = {CW * e, CW * e * N, CW * e * N * N, (cs > 0 ? (cuuint64_t)cs : vol) * e};
    cuuint32_t box[5] = {(cuuint32_t)CW, (cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return fn(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5,
              const_cast<void*>(base), dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int R, int MASK, int PM>
cudaError_t launch_tma(dim3 grid, cudaStream_t st, const TmaMaps& maps, const TmaArgs& a)
{
    constexpr size_t smem = (size_t)tma_ring_bytes<T, R, MASK>(tma_la<T, R, MASK>(), tma_lb<T, R, MASK>());
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_limit_once(attr, stencil_tma_kernel<T, R, MASK, PM>, smem);
    if (e != cudaSuccess) return e;
    stencil_tma_kernel<T, R, MASK, PM><<<grid, kTmaThreads + 32, smem, st>>>(maps, a);
    return cudaGetLastError();
}

template <typename T, int R, int PM>
cudaError_t launch_tma_masked(int mask, dim3 grid, cudaStream_t st, const TmaMaps& m, const TmaArgs& a)
{
    if constexpr (PM == PM_TLEFT) {
        switch (mask) {
        case HAS_VS: return launch_tma<T, R, HAS_VS, PM>(grid, st, m, a);
        case HAS_VS | HAS_PP: return launch_tma<T, R, HAS_VS | HAS_PP, PM>(grid, st, m, a);
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (mask) {
        case 0: return launch_tma<T, R, 0, PM>(grid, st, m, a);
        case HAS_X: return launch_tma<T, R, HAS_X, PM>(grid, st, m, a);
        case HAS_X | HAS_PREV: return launch_tma<T, R, HAS_X | HAS_PREV, PM>(grid, st, m, a);
        case HAS_X | HAS_PP: return launch_tma<T, R, HAS_X | HAS_PP, PM>(grid, st, m, a);
        case HAS_X | HAS_PREV | HAS_PP: return launch_tma<T, R, HAS_X | HAS_PREV | HAS_PP, PM>(grid, st, m, a);
        case HAS_PP: return launch_tma<T, R, HAS_PP, PM>(grid, st, m, a);
        case HAS_VS: return launch_tma<T, R, HAS_VS, PM>(grid, st, m, a);
        case HAS_VS | HAS_PP: return launch_tma<T, R, HAS_VS | HAS_PP, PM>(grid, st, m, a);
        default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace

template <typename T>
bool stencil_tma_eligible(int N)
{
    return N >= TMX && N % TMX == 0 && N % tma_ty<T>() == 0 && encode_tiled() != nullptr;
}

template <typename T>
cudaError_t launch_stencil_tma(const StencilOp& op, const StencilPass& p, const int* shift_of,
                               const double* sigma, const void* jac, const int* chunk_active,
                               int64_t n, int* err, int cn, int pmode, cudaStream_t st)
{
    const int N = op.N;
    const int R = op.order == 2 ? 1 : 2;
    if (!stencil_tma_eligible<T>(N) || cn < 1 || (pmode != PM_NONE && pmode != PM_TLEFT))
        return cudaErrorInvalidValue;
    if (p.useV != p.useSigma) return cudaErrorInvalidValue;
    const int mask = (p.x ? HAS_X : 0) | (p.prev ? HAS_PREV : 0) | (p.pp ? HAS_PP : 0) |
                     (p.useV ? HAS_VS : 0);
    constexpr int TY = tma_ty<T>();
    TmaMaps m;
    std::memset(&m, 0, sizeof(m));
    bool ok = encode_box<T>(&m.in_c, p.in, p.in_cs, N, cn, TMX, TY) &&
              encode_box<T>(&m.in_x, p.in, p.in_cs, N, cn, R, TY) &&
              encode_box<T>(&m.in_y, p.in, p.in_cs, N, cn, TMX, R);
    int k = 0;
    if (ok && p.x) ok = encode_box<T>(&m.op[k++], p.x, p.x_cs, N, cn, TMX, TY);
    if (ok && p.prev) ok = encode_box<T>(&m.op[k++], p.prev, p.prev_cs, N, cn, TMX, TY);
    if (ok && p.pp) ok = encode_box<T>(&m.op[k++], p.pp, p.pp_cs, N, cn, TMX, TY);
    if (!ok) return cudaErrorInvalidValue;
    TmaArgs a;
    a.p = p;
    a.op = op;
    a.shift_of = shift_of;
    a.sigma = sigma;
    a.jac = jac;
    a.chunk_active = chunk_active;
    a.n = n;
    a.err = err;
    const int zb = op.zb > 0 ? op.zb : 32;
    dim3 grid((unsigned)((N / TMX) * (N / TY)), (unsigned)((N + zb - 1) / zb), (unsigned)cn);
    if (pmode == PM_TLEFT)
        return R == 1 ? launch_tma_masked<T, 1, PM_TLEFT>(mask, grid, st, m, a)
                      : launch_tma_masked<T, 2, PM_TLEFT>(mask, grid, st, m, a);
    return R == 1 ? launch_tma_masked<T, 1, PM_NONE>(mask, grid, st, m, a)
                  : launch_tma_masked<T, 2, PM_NONE>(mask, grid, st, m, a);
}

template bool stencil_tma_eligible<float>(int);
template bool stencil_tma_eligible<double>(int);
template cudaError_t launch_stencil_tma<float>(const StencilOp&, const StencilPass&, const int*,
                                               const double*, const void*, const int*, int64_t,
                                               int*, int, int, cudaStream_t);
template cudaError_t launch_stencil_tma<double>(const StencilOp&, const StencilPass&, const int*,
                                                const double*, const void*, const int*, int64_t,
                                                int*, int, int, cudaStream_t);

}  // namespace evc
