// evc_stencil.cu -- matrix-free applies of the periodic finite-difference
// Hamiltonian H = -1/2 Lap_h + V and of the kinetic operator K = -1/2 Lap_h + cI
// on a block of probe columns.  One kernel serves every pass of the
// preconditioned operator C = M (H - sigma I) M (Sec. 2, Eq. negi_T):
//   * the Clenshaw steps of the Chebyshev preconditioner M = p_d(K)
//     (Sec. 6, kinetic-energy preconditioning),
//   * the shifted Hamiltonian (H - sigma_c I) with a per-column shift,
//   * the Jacobi-scaled operator diag(m) (H - sigma I) diag(m), or
//     diag(m^2) (H - sigma I) for the T^{-1}-inner-product process (Eq. lanT1),
//   * and the closing term "- beta_i q_{i-1}" of Algorithm 1.
//
// Layout: X[chunk][p][32] with p = x + N*(y + N*z).  Each thread owns one
// 16-byte vector of columns (4 FP32 or 2 FP64 probes) of one (x, y) line and
// marches along z keeping the z-neighbours in a register window.  The loads
// of plane z + D (in-plane neighbours, the next window plane, the pointwise
// operands) are issued as asynchronous 16-byte copies (cp.async) into the
// thread's own shared-memory slots while plane z is computed, so the bytes
// in flight are held by shared memory rather than registers.  The pass is
// HBM-bound: it streams the operand once and the pointwise operands once.
#include "evc_internal.cuh"

#include <cstring>

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
__device__ __forceinline__ Pack<T> ld_pack(const Pack<T>* p)
{
    typename Vec16<T>::type t = *reinterpret_cast<const typename Vec16<T>::type*>(p);
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

constexpr int ZB = 32;     // z planes per block unless tuned (StencilOp::zb)
constexpr int STH = 128;   // threads per block
constexpr int DEPTH = 3;   // planes of loads in flight ahead of the one computed

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    // 16-byte asynchronous copy global -> shared, cached in L1 (neighbour reuse)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N_>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N_) : "memory"); }

struct KArgs {
    StencilPass p;
    StencilOp op;
    const int* shift_of;
    const double* sigma;
    const void* jac;
    const int* chunk_active;
    int64_t n;
};

// Operand set of a pass, a compile-time mask so that absent operands cost
// neither instructions nor registers.
enum { HAS_X = 1, HAS_PREV = 2, HAS_PP = 4, HAS_VS = 8 };

template <typename T, int R, int PM, int MASK>
__global__ void __launch_bounds__(STH)
stencil_pass_kernel(KArgs a)
{
    constexpr bool JAC = PM == PM_JACOBI;    // operand scaled by m on load
    constexpr bool ROWS = PM != PM_NONE;     // output scaled (m, or m^2 = T)
    constexpr int W = 16 / sizeof(T);        // columns per thread
    constexpr int LPP = CW / W;              // threads per grid point
    constexpr int TX = 8;                    // points per block along x
    constexpr int TY = STH / LPP / TX;       // points per block along y
    constexpr bool X = MASK & HAS_X, PREV = MASK & HAS_PREV, PP = MASK & HAS_PP,
                   VS = MASK & HAS_VS;
    // loads per plane: 4R in-plane neighbours, the next window plane, pointwise operands
    constexpr int NL = 4 * R + 1 + (X ? 1 : 0) + (PREV ? 1 : 0) + (PP ? 1 : 0);
    constexpr int UC = 4 * R, UX = UC + 1, UP = UX + (X ? 1 : 0), UPP = UP + (PREV ? 1 : 0);
    const int ch = blockIdx.z;
    if (!a.chunk_active[ch]) return;
    extern __shared__ __align__(16) unsigned char st_raw[];
    Pack<T>* slots = reinterpret_cast<Pack<T>*>(st_raw);      // [DEPTH+1][NL][STH]
    // per-column constants of this chunk, shared by the block
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
    __syncthreads();
    const int N = a.op.N;
    const int lane = threadIdx.x % LPP;
    const int pt = threadIdx.x / LPP;
    const int tilesX = (N + TX - 1) / TX;
    const int x = (blockIdx.x % tilesX) * TX + pt % TX;
    const int y = (blockIdx.x / tilesX) * TY + pt / TX;
    if (x >= N || y >= N) return;            // no block-level barriers below
    const int zb = a.op.zb > 0 ? a.op.zb : ZB;
    const int z0 = blockIdx.y * zb;
    const int z1 = min(z0 + zb, N);
    const int64_t n = a.n;
    const int64_t NN = (int64_t)N * N;

    const Pack<T>* in = reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.in) + ch * a.p.in_cs) + lane;
    const Pack<T>* xv = X ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.x) + ch * a.p.x_cs) + lane : nullptr;
    const Pack<T>* pv = PREV ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.prev) + ch * a.p.prev_cs) + lane : nullptr;
    const Pack<T>* ppv = PP ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.pp) + ch * a.p.pp_cs) + lane : nullptr;
    Pack<T>* out = reinterpret_cast<Pack<T>*>(static_cast<T*>(a.p.out) + ch * a.p.out_cs) + lane;
    const T* __restrict__ V = static_cast<const T*>(a.op.V);
    const T* __restrict__ jac = static_cast<const T*>(a.jac);
    const int sbase = lane * W;

    // wrapped in-plane neighbour offsets (points), fixed along the z march
    const int xm1 = x == 0 ? N - 1 : x - 1, xp1 = x == N - 1 ? 0 : x + 1;
    const int ym1 = y == 0 ? N - 1 : y - 1, yp1 = y == N - 1 ? 0 : y + 1;
    const int64_t cxy = x + (int64_t)N * y;
    int64_t nbo[4 * R];
    nbo[0] = xm1 + (int64_t)N * y;
    nbo[1] = xp1 + (int64_t)N * y;
    nbo[2] = x + (int64_t)N * ym1;
    nbo[3] = x + (int64_t)N * yp1;
    if (R == 2) {
        nbo[4 % (4 * R)] = (x + N - 2) % N + (int64_t)N * y;
        nbo[5 % (4 * R)] = (x + 2) % N + (int64_t)N * y;
        nbo[6 % (4 * R)] = x + (int64_t)N * ((y + N - 2) % N);
        nbo[7 % (4 * R)] = x + (int64_t)N * ((y + 2) % N);
    }
    auto slot = [&](int stage, int u) -> Pack<T>* {
        return slots + ((size_t)stage * NL + u) * STH + threadIdx.x;
    };
    auto jscale = [&](Pack<T>& v, int64_t q) {
        if (JAC) {
#pragma unroll
            for (int w = 0; w < W; ++w) v.v[w] *= __ldg(jac + (int64_t)s_shift[sbase + w] * n + q);
        }
    };
    // issue the loads of plane zz into stage st (one commit group per plane;
    // an empty group past the end keeps the group count uniform)
    // source pointers of the next plane to issue, advanced one plane per issue
    const int64_t pstep = NN * LPP;
    const Pack<T>* src_nb[4 * R];
#pragma unroll
    for (int u = 0; u < 4 * R; ++u) src_nb[u] = in + (nbo[u] + NN * z0) * LPP;
    const Pack<T>* src_x = X ? xv + (cxy + NN * z0) * LPP : nullptr;
    const Pack<T>* src_p = PREV ? pv + (cxy + NN * z0) * LPP : nullptr;
    const Pack<T>* src_pp = PP ? ppv + (cxy + NN * z0) * LPP : nullptr;
    auto issue = [&](int zz, int st) {
        if (zz < z1) {
#pragma unroll
            for (int u = 0; u < 4 * R; ++u) {
                cp_async16(slot(st, u), src_nb[u]);
                src_nb[u] += pstep;
            }
            if (zz + 1 < z1) cp_async16(slot(st, UC), in + (cxy + NN * ((zz + 1 + R) % N)) * LPP);
            if (X) { cp_async16(slot(st, UX), src_x); src_x += pstep; }
            if (PREV) { cp_async16(slot(st, UP), src_p); src_p += pstep; }
            if (PP) { cp_async16(slot(st, UPP), src_pp); src_pp += pstep; }
        }
        cp_async_commit();
    };

    Pack<T> win[2 * R + 1];
#pragma unroll
    for (int o = -R; o <= R; ++o) {
        const int64_t q = cxy + NN * (((z0 + o) % N + N) % N);
        win[o + R] = ldg_pack(in + q * LPP);
        jscale(win[o + R], q);
    }
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) issue(z0 + d, d);

    const T k1 = (T)a.p.k1;
    const T c1 = (T)a.op.c1, c2 = (T)a.op.c2;
    const T dg = (T)(a.p.k1 * a.op.cd + a.p.k0);
    const T a2 = (T)a.p.a2;

    for (int z = z0; z < z1; ++z) {
        const int stg = (z - z0) % (DEPTH + 1);
        issue(z + DEPTH, (z - z0 + DEPTH) % (DEPTH + 1));
        cp_async_wait<DEPTH>();                  // plane z has landed (own copies)
        const int64_t rowz = NN * z;
        const int64_t p = cxy + rowz;
        Pack<T> nb[4 * R];
#pragma unroll
        for (int u = 0; u < 4 * R; ++u) {
            nb[u] = *slot(stg, u);
            jscale(nb[u], nbo[u] + rowz);
        }
        const T vp = VS ? __ldg(V + p) : (T)0;
        T mp[W];
        if (ROWS) {
#pragma unroll
            for (int w = 0; w < W; ++w) mp[w] = __ldg(jac + (int64_t)s_shift[sbase + w] * n + p);
        }
        const Pack<T> sig = s_sig[lane], insc = s_insc[lane];
        Pack<T> res;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            T off = c1 * (nb[0].v[w] + nb[1].v[w] + nb[2].v[w] + nb[3].v[w] +
                          win[R - 1].v[w] + win[R + 1].v[w]);
            if (R == 2)
                off += c2 * (nb[4 % (4 * R)].v[w] + nb[5 % (4 * R)].v[w] + nb[6 % (4 * R)].v[w] +
                             nb[7 % (4 * R)].v[w] + win[0].v[w] + win[2 * R].v[w]);
            T st = k1 * off + (dg + vp - sig.v[w]) * win[R].v[w];
            if (ROWS) st *= mp[w];
            res.v[w] = insc.v[w] * st;
        }
        if (X) {
            const Pack<T> t = *slot(stg, UX), c = s_a0s[lane];
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] += c.v[w] * t.v[w];
        }
        if (PREV) {
            const Pack<T> t = *slot(stg, UP);
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] -= a2 * t.v[w];
        }
        if (PP) {
            const Pack<T> t = *slot(stg, UPP), c = s_ppc[lane];
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] -= c.v[w] * t.v[w];
        }
        st_pack(out + p * LPP, res);
        if (z + 1 < z1) {
            Pack<T> nxt = *slot(stg, UC);
            jscale(nxt, cxy + NN * ((z + 1 + R) % N));
#pragma unroll
            for (int o = 0; o < 2 * R; ++o) win[o] = win[o + 1];
            win[2 * R] = nxt;
        }
    }
    cp_async_wait<0>();
}

// Patch variant of the same pass (no operand scaling; PM_TLEFT scales the
// output rows by T = m^2 for the T^{-1}-inner-product process): each thread owns the
// same 16-byte column vector of a PX x PY patch of (x, y) points and marches
// them along z together.  Neighbours that fall inside the patch come from the
// thread's own register window; only the 2R(PX + PY) points around the patch
// are loaded.  The pass is bound by the L1 pipe (one cp.async and one
// shared-memory read per loaded vector), so a 2 x 2 patch cuts the loads per
// output of the 7-point stencil from 4R + 1 to R(PX + PY)/2 + 1 plus the
// pointwise operands.  Per-point arithmetic and summation order are those of
// stencil_pass_kernel.  N must be a multiple of PX and PY.
constexpr int STP1 = 128;  // threads per block of the patch variant, 7-point
constexpr int STP2 = 128;  // threads per block of the patch variant, 13-point

template <int R>
__host__ __device__ constexpr int patch_threads()
{
    return R == 1 ? STP1 : STP2;
}
constexpr int DMAXP = 3;   // planes of loads in flight, patch variant (at most)
constexpr int PTW = 8;     // patch-variant block tile width (points along x)

// Planes in flight of one patch-kernel instance (slots: NL per plane per
// thread).  7-point (R = 1): DMAXP, or fewer when the slots would not fit one
// block of 220 KB.  13-point (R = 2): as many as let two blocks share an SM
// (113 KB each) -- measured 23% faster than a deeper pipeline with one block --
// falling back to the one-block rule when not even one plane allows that.  For
// R = 1 the one-block rule measured 1% ahead on one stream and 4% ahead with
// four concurrent chunk groups (52.3 against 54.3 ms per 64^3 count).
template <int R, int MASK, int PX, int PY>
__host__ __device__ constexpr int patch_depth()
{
    constexpr int nl = 2 * R * (PX + PY) +
                       PX * PY * (1 + ((MASK & HAS_X) ? 1 : 0) + ((MASK & HAS_PREV) ? 1 : 0) +
                                  ((MASK & HAS_PP) ? 1 : 0));
    constexpr int two = 113 * 1024 / (nl * patch_threads<R>() * 16) - 1;
    constexpr int one = 220 * 1024 / (nl * patch_threads<R>() * 16) - 1;
    constexpr int fit = (R == 2 && two > 0) ? two : one;
    return fit < DMAXP ? fit : DMAXP;
}

template <typename T, int R, int MASK, int PX, int PY, int PM>
__global__ void __launch_bounds__(patch_threads<R>())
stencil_patch_kernel(KArgs a)
{
    static_assert(PM == PM_NONE || PM == PM_TLEFT, "the patch pass scales no operand");
    constexpr bool ROWS = PM == PM_TLEFT;
    constexpr int STP = patch_threads<R>();
    constexpr int DEPTHP = patch_depth<R, MASK, PX, PY>();
    static_assert(DEPTHP >= 1, "patch kernel slots do not fit shared memory");
    constexpr int W = 16 / sizeof(T);
    constexpr int LPP = CW / W;
    constexpr int NPT = PX * PY;                 // points per thread
    constexpr int TXP = PTW / PX;                // patches per block along x
    constexpr int TYP = STP / LPP / TXP;         // patches per block along y
    constexpr bool X = MASK & HAS_X, PREV = MASK & HAS_PREV, PP = MASK & HAS_PP,
                   VS = MASK & HAS_VS;
    constexpr int NBX = 2 * R * PY, NBY = 2 * R * PX, NB = NBX + NBY;
    constexpr int NOP = (X ? 1 : 0) + (PREV ? 1 : 0) + (PP ? 1 : 0);
    constexpr int UC = NB;                       // next window plane of each point
    constexpr int UO = NB + NPT;                 // operands: [op][point]
    constexpr int NL = NB + NPT * (1 + NOP);
    const int ch = blockIdx.z;
    if (!a.chunk_active[ch]) return;
    extern __shared__ __align__(16) unsigned char st_raw[];
    Pack<T>* slots = reinterpret_cast<Pack<T>*>(st_raw);      // [DEPTHP+1][NL][STP]
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
    __syncthreads();
    const int N = a.op.N;
    const int lane = threadIdx.x % LPP;
    const int pt = threadIdx.x / LPP;
    const T* __restrict__ jac = static_cast<const T*>(a.jac);
    const int64_t n = a.n;
    const int tilesX = (N + TXP * PX - 1) / (TXP * PX);
    const int x = (blockIdx.x % tilesX) * (TXP * PX) + (pt % TXP) * PX;
    const int y = (blockIdx.x / tilesX) * (TYP * PY) + (pt / TXP) * PY;
    if (x >= N || y >= N) return;            // whole patch outside (N % PX == N % PY == 0)
    const int zb = a.op.zb > 0 ? a.op.zb : ZB;
    const int z0 = blockIdx.y * zb;
    const int z1 = min(z0 + zb, N);
    const int64_t NN = (int64_t)N * N;
    const Pack<T>* in = reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.in) + ch * a.p.in_cs) + lane;
    const Pack<T>* xv = X ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.x) + ch * a.p.x_cs) + lane : nullptr;
    const Pack<T>* pv = PREV ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.prev) + ch * a.p.prev_cs) + lane : nullptr;
    const Pack<T>* ppv = PP ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.pp) + ch * a.p.pp_cs) + lane : nullptr;
    Pack<T>* out = reinterpret_cast<Pack<T>*>(static_cast<T*>(a.p.out) + ch * a.p.out_cs) + lane;
    const T* __restrict__ V = static_cast<const T*>(a.op.V);
    auto wrap = [&](int v) { return v < 0 ? v + N : (v >= N ? v - N : v); };

    int64_t cxy[NPT];
#pragma unroll
    for (int b = 0; b < PY; ++b)
#pragma unroll
        for (int q = 0; q < PX; ++q) cxy[b * PX + q] = (x + q) + (int64_t)N * (y + b);
    // the points around the patch: per row, offsets -R..-1 and PX..PX+R-1 in
    // x; per column, the same in y (slot d < R: offset d - R, else d - R + P)
    const int64_t pstep = NN * LPP;
    const Pack<T>* src_nb[NB];
#pragma unroll
    for (int b = 0; b < PY; ++b)
#pragma unroll
        for (int d = 0; d < 2 * R; ++d) {
            const int o = d < R ? d - R : PX + d - R;
            src_nb[b * 2 * R + d] = in + (wrap(x + o) + (int64_t)N * (y + b) + NN * z0) * LPP;
        }
#pragma unroll
    for (int q = 0; q < PX; ++q)
#pragma unroll
        for (int d = 0; d < 2 * R; ++d) {
            const int o = d < R ? d - R : PY + d - R;
            src_nb[NBX + q * 2 * R + d] = in + ((x + q) + (int64_t)N * wrap(y + o) + NN * z0) * LPP;
        }
    auto slot = [&](int stage, int u) -> Pack<T>* {
        return slots + ((size_t)stage * NL + u) * STP + threadIdx.x;
    };
    auto issue = [&](int zz, int st) {
        if (zz < z1) {
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                cp_async16(slot(st, u), src_nb[u]);
                src_nb[u] += pstep;
            }
            if (zz + 1 < z1) {
                const int64_t zc = NN * ((zz + 1 + R) % N);
#pragma unroll
                for (int q = 0; q < NPT; ++q) cp_async16(slot(st, UC + q), in + (cxy[q] + zc) * LPP);
            }
            const int64_t zo = NN * zz;
            int k = 0;
            if (X) {
#pragma unroll
                for (int q = 0; q < NPT; ++q) cp_async16(slot(st, UO + k * NPT + q), xv + (cxy[q] + zo) * LPP);
                ++k;
            }
            if (PREV) {
#pragma unroll
                for (int q = 0; q < NPT; ++q) cp_async16(slot(st, UO + k * NPT + q), pv + (cxy[q] + zo) * LPP);
                ++k;
            }
            if (PP) {
#pragma unroll
                for (int q = 0; q < NPT; ++q) cp_async16(slot(st, UO + k * NPT + q), ppv + (cxy[q] + zo) * LPP);
            }
        }
        cp_async_commit();
    };

    Pack<T> win[2 * R + 1][NPT];
#pragma unroll
    for (int o = -R; o <= R; ++o) {
        const int64_t zq = NN * (((z0 + o) % N + N) % N);
#pragma unroll
        for (int q = 0; q < NPT; ++q) win[o + R][q] = ldg_pack(in + (cxy[q] + zq) * LPP);
    }
#pragma unroll
    for (int d = 0; d < DEPTHP; ++d) issue(z0 + d, d);

    const T k1 = (T)a.p.k1;
    const T c1 = (T)a.op.c1, c2 = (T)a.op.c2;
    const T dg = (T)(a.p.k1 * a.op.cd + a.p.k0);
    const T a2 = (T)a.p.a2;

    for (int z = z0; z < z1; ++z) {
        const int stg = (z - z0) % (DEPTHP + 1);
        issue(z + DEPTHP, (z - z0 + DEPTHP) % (DEPTHP + 1));
        cp_async_wait<DEPTHP>();
        const int64_t rowz = NN * z;
        Pack<T> nb[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) nb[u] = *slot(stg, u);
        const Pack<T> sig = s_sig[lane], insc = s_insc[lane], a0c = s_a0s[lane], ppcc = s_ppc[lane];
#pragma unroll
        for (int b = 0; b < PY; ++b) {
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                const int pp_ = b * PX + q;
                // value of the plane-z point at offset (ox, oy) from point (q, b)
                auto nbv = [&](int ox, int oy) -> const Pack<T>& {
                    const int xx = q + ox, yy = b + oy;
                    if (oy == 0) {
                        if (xx >= 0 && xx < PX) return win[R][b * PX + xx];
                        return nb[b * 2 * R + (xx < 0 ? xx + R : R + xx - PX)];
                    }
                    if (yy >= 0 && yy < PY) return win[R][yy * PX + q];
                    return nb[NBX + q * 2 * R + (yy < 0 ? yy + R : R + yy - PY)];
                };
                const T vp = VS ? __ldg(V + cxy[pp_] + rowz) : (T)0;
                Pack<T> res;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    T off = c1 * (nbv(-1, 0).v[w] + nbv(1, 0).v[w] + nbv(0, -1).v[w] +
                                  nbv(0, 1).v[w] + win[R - 1][pp_].v[w] + win[R + 1][pp_].v[w]);
                    if (R == 2)
                        off += c2 * (nbv(-2, 0).v[w] + nbv(2, 0).v[w] + nbv(0, -2).v[w] +
                                     nbv(0, 2).v[w] + win[0][pp_].v[w] + win[2 * R][pp_].v[w]);
                    T stv = k1 * off + (dg + vp - sig.v[w]) * win[R][pp_].v[w];
                    if (ROWS)
                        stv *= __ldg(jac + (int64_t)s_shift[lane * W + w] * n + cxy[pp_] + rowz);
                    res.v[w] = insc.v[w] * stv;
                }
                int k = 0;
                if (X) {
                    const Pack<T> t = *slot(stg, UO + (k++) * NPT + pp_);
#pragma unroll
                    for (int w = 0; w < W; ++w) res.v[w] += a0c.v[w] * t.v[w];
                }
                if (PREV) {
                    const Pack<T> t = *slot(stg, UO + (k++) * NPT + pp_);
#pragma unroll
                    for (int w = 0; w < W; ++w) res.v[w] -= a2 * t.v[w];
                }
                if (PP) {
                    const Pack<T> t = *slot(stg, UO + (k++) * NPT + pp_);
#pragma unroll
                    for (int w = 0; w < W; ++w) res.v[w] -= ppcc.v[w] * t.v[w];
                }
                st_pack(out + (cxy[pp_] + rowz) * LPP, res);
            }
        }
        if (z + 1 < z1) {
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                const Pack<T> nxt = *slot(stg, UC + q);
#pragma unroll
                for (int o = 0; o < 2 * R; ++o) win[o][q] = win[o + 1][q];
                win[2 * R][q] = nxt;
            }
        }
    }
    cp_async_wait<0>();
}

template <typename T, int R, int MASK, int PX, int PY, int PM = PM_NONE>
void launch_patch(dim3 grid, cudaStream_t st, const KArgs& a)
{
    constexpr int NB = 2 * R * (PX + PY);
    constexpr int NOP = ((MASK & HAS_X) ? 1 : 0) + ((MASK & HAS_PREV) ? 1 : 0) + ((MASK & HAS_PP) ? 1 : 0);
    constexpr int STP = patch_threads<R>();
    constexpr size_t smem =
        (size_t)(patch_depth<R, MASK, PX, PY>() + 1) * (NB + PX * PY * (1 + NOP)) * STP * 16;
    // a failure here shows as the launch's error
    static std::atomic<uint64_t> attr{0};
    smem_limit_once(attr, stencil_patch_kernel<T, R, MASK, PX, PY, PM>, smem);
    stencil_patch_kernel<T, R, MASK, PX, PY, PM><<<grid, STP, smem, st>>>(a);
}

// The operand sets of the T-scaled Lanczos step (V and the shift, with or
// without q_{i-1}).
template <typename T, int R, int PX, int PY>
bool launch_patch_masked_tl(int mask, dim3 grid, cudaStream_t st, const KArgs& a)
{
    switch (mask) {
    case HAS_VS: launch_patch<T, R, HAS_VS, PX, PY, PM_TLEFT>(grid, st, a); break;
    case HAS_VS | HAS_PP: launch_patch<T, R, HAS_VS | HAS_PP, PX, PY, PM_TLEFT>(grid, st, a); break;
    default:
        return false;
    }
    return true;
}

template <typename T, int R, int PX, int PY>
bool launch_patch_masked(int mask, dim3 grid, cudaStream_t st, const KArgs& a)
{
    switch (mask) {
    case 0: launch_patch<T, R, 0, PX, PY>(grid, st, a); break;
    case HAS_X: launch_patch<T, R, HAS_X, PX, PY>(grid, st, a); break;
    case HAS_X | HAS_PREV: launch_patch<T, R, HAS_X | HAS_PREV, PX, PY>(grid, st, a); break;
    case HAS_X | HAS_PP: launch_patch<T, R, HAS_X | HAS_PP, PX, PY>(grid, st, a); break;
    case HAS_X | HAS_PREV | HAS_PP: launch_patch<T, R, HAS_X | HAS_PREV | HAS_PP, PX, PY>(grid, st, a); break;
    case HAS_PP: launch_patch<T, R, HAS_PP, PX, PY>(grid, st, a); break;
    case HAS_VS: launch_patch<T, R, HAS_VS, PX, PY>(grid, st, a); break;
    case HAS_VS | HAS_PP: launch_patch<T, R, HAS_VS | HAS_PP, PX, PY>(grid, st, a); break;
    default:
        return false;
    }
    return true;
}

template <int R, int MASK>
constexpr int stencil_loads()
{
    return 4 * R + 1 + ((MASK & HAS_X) ? 1 : 0) + ((MASK & HAS_PREV) ? 1 : 0) +
           ((MASK & HAS_PP) ? 1 : 0);
}

template <typename T, int R, int PM, int MASK>
void launch_one(dim3 grid, cudaStream_t st, const KArgs& a)
{
    constexpr size_t smem = (size_t)(DEPTH + 1) * stencil_loads<R, MASK>() * STH * 16;
    static std::atomic<uint64_t> attr{0};
    smem_limit_once(attr, stencil_pass_kernel<T, R, PM, MASK>, smem);
    stencil_pass_kernel<T, R, PM, MASK><<<grid, STH, smem, st>>>(a);
}

template <typename T, int R, int PM>
bool launch_masked(int mask, dim3 grid, cudaStream_t st, const KArgs& a)
{
    switch (mask) {
    case 0: launch_one<T, R, PM, 0>(grid, st, a); break;
    case HAS_X: launch_one<T, R, PM, HAS_X>(grid, st, a); break;
    case HAS_X | HAS_PREV: launch_one<T, R, PM, HAS_X | HAS_PREV>(grid, st, a); break;
    case HAS_X | HAS_PP: launch_one<T, R, PM, HAS_X | HAS_PP>(grid, st, a); break;
    case HAS_X | HAS_PREV | HAS_PP: launch_one<T, R, PM, HAS_X | HAS_PREV | HAS_PP>(grid, st, a); break;
    case HAS_PP: launch_one<T, R, PM, HAS_PP>(grid, st, a); break;
    case HAS_VS: launch_one<T, R, PM, HAS_VS>(grid, st, a); break;
    case HAS_VS | HAS_PP: launch_one<T, R, PM, HAS_VS | HAS_PP>(grid, st, a); break;
    default:
        return false;   // not an operand set the library issues
    }
    return true;
}

// The operand sets of the diagonally preconditioned passes: the Lanczos step
// (V and the shift, with or without q_{i-1}).
template <typename T, int R, int PM>
bool launch_masked_diag(int mask, dim3 grid, cudaStream_t st, const KArgs& a)
{
    switch (mask) {
    case HAS_VS: launch_one<T, R, PM, HAS_VS>(grid, st, a); break;
    case HAS_VS | HAS_PP: launch_one<T, R, PM, HAS_VS | HAS_PP>(grid, st, a); break;
    default:
        return false;
    }
    return true;
}

}  // namespace

template <typename T>
cudaError_t launch_stencil_pass(const StencilOp& op, const Run& r, const StencilPass& p,
                                int pmode, cudaStream_t st)
{
    constexpr int W = 16 / sizeof(T);
    constexpr int LPP = CW / W;
    constexpr int TX = 8;
    constexpr int TY = STH / LPP / TX;
    // a chunk range is a view: every per-chunk pointer moves to chunk c0 and
    // the kernels see chunks 0 .. cn-1 of it (Jacobi scales and V are indexed
    // by shift and point, not by chunk)
    const int c0 = op.cn > 0 ? op.c0 : 0;
    const int cn = op.cn > 0 ? op.cn : r.nchunk;
    if (c0 < 0 || c0 + cn > r.nchunk) return cudaErrorInvalidValue;
    auto at = [&](const void* q, int64_t cs) -> const void* {
        return q ? static_cast<const void*>(static_cast<const T*>(q) + (int64_t)c0 * cs) : q;
    };
    auto atc = [&](const double* q) { return q ? q + (int64_t)c0 * CW : q; };
    KArgs a;
    a.p = p;
    a.p.in = at(p.in, p.in_cs);
    a.p.x = at(p.x, p.x_cs);
    a.p.prev = at(p.prev, p.prev_cs);
    a.p.pp = at(p.pp, p.pp_cs);
    a.p.out = const_cast<void*>(at(p.out, p.out_cs));
    a.p.insc = atc(p.insc);
    a.p.xs = atc(p.xs);
    a.p.ppc = atc(p.ppc);
    a.op = op;
    a.shift_of = r.shift_of + (int64_t)c0 * CW;
    a.sigma = atc(r.sigma);
    a.jac = r.jac;
    a.chunk_active = r.chunk_active + c0;
    a.n = r.n;
    const int N = op.N;
    const int zb = op.zb > 0 ? op.zb : ZB;
    dim3 grid(((N + TX - 1) / TX) * ((N + TY - 1) / TY), (N + zb - 1) / zb, cn);
    // V and the per-column shift always enter together (the H - sigma I pass)
    if (p.useV != p.useSigma) return cudaErrorInvalidValue;
    const int mask = (p.x ? HAS_X : 0) | (p.prev ? HAS_PREV : 0) | (p.pp ? HAS_PP : 0) |
                     (p.useV ? HAS_VS : 0);
    bool ok;
    if (pmode != PM_JACOBI && op.patch == 3 && stencil_tma_eligible<T>(N))
        return launch_stencil_tma<T>(op, a.p, a.shift_of, a.sigma, a.jac, a.chunk_active, a.n, r.err,
                                     cn, pmode, st);
    if (pmode != PM_JACOBI && op.patch >= 2 && N % 2 == 0) {
        // 2 x 2 patches: PTW x (2 TYP) points per block
        const int TYP = (op.order == 2 ? patch_threads<1>() : patch_threads<2>()) / LPP / (PTW / 2);
        dim3 pg(((N + PTW - 1) / PTW) * ((N + 2 * TYP - 1) / (2 * TYP)), (N + zb - 1) / zb, cn);
        if (pmode == PM_TLEFT)
            ok = op.order == 2 ? launch_patch_masked_tl<T, 1, 2, 2>(mask, pg, st, a)
                               : launch_patch_masked_tl<T, 2, 2, 2>(mask, pg, st, a);
        else
            ok = op.order == 2 ? launch_patch_masked<T, 1, 2, 2>(mask, pg, st, a)
                               : launch_patch_masked<T, 2, 2, 2>(mask, pg, st, a);
        if (!ok) return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (pmode == PM_NONE)
        ok = op.order == 2 ? launch_masked<T, 1, PM_NONE>(mask, grid, st, a)
                           : launch_masked<T, 2, PM_NONE>(mask, grid, st, a);
    else if (pmode == PM_JACOBI)
        ok = op.order == 2 ? launch_masked_diag<T, 1, PM_JACOBI>(mask, grid, st, a)
                           : launch_masked_diag<T, 2, PM_JACOBI>(mask, grid, st, a);
    else if (pmode == PM_TLEFT)
        ok = op.order == 2 ? launch_masked_diag<T, 1, PM_TLEFT>(mask, grid, st, a)
                           : launch_masked_diag<T, 2, PM_TLEFT>(mask, grid, st, a);
    else
        ok = false;
    if (!ok) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template cudaError_t launch_stencil_pass<float>(const StencilOp&, const Run&, const StencilPass&,
                                                int, cudaStream_t);
template cudaError_t launch_stencil_pass<double>(const StencilOp&, const Run&, const StencilPass&,
                                                 int, cudaStream_t);

}  // namespace evc
