// evc_stencil.cu -- matrix-free applies of the periodic finite-difference
// Hamiltonian H = -1/2 Lap_h + V and of the kinetic operator K = -1/2 Lap_h + cI
// on a block of probe columns.  One kernel serves every pass of the
// preconditioned operator C = M (H - sigma I) M (Sec. 2, Eq. negi_T):
//   * the Clenshaw steps of the Chebyshev preconditioner M = p_d(K)
//     (Sec. 6, kinetic-energy preconditioning),
//   * the shifted Hamiltonian (H - sigma_c I) with a per-column shift,
//   * the Jacobi-scaled operator diag(m) (H - sigma I) diag(m),
//   * and the closing term "- beta_i q_{i-1}" of Algorithm 1.
//
// Layout: X[chunk][p][32] with p = x + N*(y + N*z).  Each thread owns one
// 16-byte vector of columns (4 FP32 or 2 FP64 probes) of one (x, y) line and
// marches along z keeping the z-neighbours in a register window; x/y
// neighbours come through L1.  The pass is HBM-bound: it streams the operand
// once and the pointwise operands once.
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

constexpr int TX = 8;     // points per block along x
constexpr int ZB = 16;    // z planes per block

struct KArgs {
    StencilPass p;
    StencilOp op;
    const int* shift_of;
    const double* sigma;
    const void* jac;
    const int* chunk_active;
    int64_t n;
};

template <typename T, int R, bool JAC>
__global__ void __launch_bounds__(kThreads, R == 1 ? 4 : 3)
stencil_pass_kernel(KArgs a)
{
    constexpr int W = 16 / sizeof(T);        // columns per thread
    constexpr int LPP = CW / W;              // threads per grid point
    constexpr int TY = kThreads / LPP / TX;  // points per block along y
    const int ch = blockIdx.z;
    if (!a.chunk_active[ch]) return;
    // per-column constants of this chunk, shared by the block
    __shared__ Pack<T> s_sig[LPP], s_insc[LPP], s_a0s[LPP], s_ppc[LPP];
    __shared__ int s_shift[CW];
    if (threadIdx.x < CW) {
        const int c = ch * CW + threadIdx.x;
        const int l = threadIdx.x / W, w = threadIdx.x % W;
        s_sig[l].v[w] = a.p.useSigma ? (T)a.sigma[c] : (T)0;
        s_insc[l].v[w] = a.p.insc ? (T)a.p.insc[c] : (T)1;
        s_a0s[l].v[w] = (T)(a.p.a0 * (a.p.xs ? a.p.xs[c] : 1.0));
        s_ppc[l].v[w] = a.p.ppc ? (T)a.p.ppc[c] : (T)0;
        s_shift[threadIdx.x] = JAC ? a.shift_of[c] : 0;
    }
    __syncthreads();
    const int N = a.op.N;
    const int lane = threadIdx.x % LPP;
    const int pt = threadIdx.x / LPP;
    const int tilesX = (N + TX - 1) / TX;
    const int x = (blockIdx.x % tilesX) * TX + pt % TX;
    const int y = (blockIdx.x / tilesX) * TY + pt / TX;
    if (x >= N || y >= N) return;            // no block-level barriers below
    const int z0 = blockIdx.y * ZB;
    const int z1 = min(z0 + ZB, N);
    const int64_t n = a.n;

    const Pack<T>* __restrict__ in = reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.in) + ch * a.p.in_cs) + lane;
    const Pack<T>* __restrict__ xv = a.p.x ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.x) + ch * a.p.x_cs) + lane : nullptr;
    const Pack<T>* pv = a.p.prev ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.prev) + ch * a.p.prev_cs) + lane : nullptr;
    const Pack<T>* __restrict__ ppv = a.p.pp ? reinterpret_cast<const Pack<T>*>(
        static_cast<const T*>(a.p.pp) + ch * a.p.pp_cs) + lane : nullptr;
    Pack<T>* out = reinterpret_cast<Pack<T>*>(static_cast<T*>(a.p.out) + ch * a.p.out_cs) + lane;
    const T* __restrict__ V = static_cast<const T*>(a.op.V);
    const T* __restrict__ jac = static_cast<const T*>(a.jac);

    const T k1 = (T)a.p.k1;
    const T c1 = (T)a.op.c1, c2 = (T)a.op.c2;
    const T dg = (T)(a.p.k1 * a.op.cd + a.p.k0);
    const T a2 = (T)a.p.a2;

    // wrapped in-plane neighbour coordinates
    const int xm1 = x == 0 ? N - 1 : x - 1, xp1 = x == N - 1 ? 0 : x + 1;
    const int ym1 = y == 0 ? N - 1 : y - 1, yp1 = y == N - 1 ? 0 : y + 1;
    const int xm2 = (x + N - 2) % N, xp2 = (x + 2) % N;
    const int ym2 = (y + N - 2) % N, yp2 = (y + 2) % N;
    const int64_t NN = (int64_t)N * N;
    const int64_t cxy = x + (int64_t)N * y;
    const int64_t oxm1 = xm1 + (int64_t)N * y, oxp1 = xp1 + (int64_t)N * y;
    const int64_t oym1 = x + (int64_t)N * ym1, oyp1 = x + (int64_t)N * yp1;
    const int64_t oxm2 = xm2 + (int64_t)N * y, oxp2 = xp2 + (int64_t)N * y;
    const int64_t oym2 = x + (int64_t)N * ym2, oyp2 = x + (int64_t)N * yp2;
    const int sbase = lane * W;

    auto load = [&](int64_t q) -> Pack<T> {
        Pack<T> v = ldg_pack(in + q * LPP);
        if (JAC) {
#pragma unroll
            for (int w = 0; w < W; ++w) v.v[w] *= __ldg(jac + (int64_t)s_shift[sbase + w] * n + q);
        }
        return v;
    };

    Pack<T> win[2 * R + 1];
#pragma unroll
    for (int o = -R; o <= R; ++o) {
        const int zz = ((z0 + o) % N + N) % N;
        win[o + R] = load(cxy + NN * zz);
    }

    for (int z = z0; z < z1; ++z) {
        const int64_t rowz = NN * z;
        const int64_t p = cxy + rowz;
        // every load of this plane first: they are independent
        Pack<T> nb[4 * R];
        nb[0] = load(oxm1 + rowz);
        nb[1] = load(oxp1 + rowz);
        nb[2] = load(oym1 + rowz);
        nb[3] = load(oyp1 + rowz);
        if (R == 2) {
            nb[4 % (4 * R)] = load(oxm2 + rowz);
            nb[5 % (4 * R)] = load(oxp2 + rowz);
            nb[6 % (4 * R)] = load(oym2 + rowz);
            nb[7 % (4 * R)] = load(oyp2 + rowz);
        }
        const bool more = z + 1 < z1;
        Pack<T> nxt;
        if (more) nxt = load(cxy + NN * ((z + 1 + R) % N));
        Pack<T> tx, tp, tpp;
        if (xv) tx = ldg_pack(xv + p * LPP);
        if (pv) tp = ld_pack(pv + p * LPP);
        if (ppv) tpp = ldg_pack(ppv + p * LPP);
        const T vp = a.p.useV ? __ldg(V + p) : (T)0;
        T mp[W];
        if (JAC) {
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
            if (JAC) st *= mp[w];
            res.v[w] = insc.v[w] * st;
        }
        if (xv) {
            const Pack<T> a0s = s_a0s[lane];
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] += a0s.v[w] * tx.v[w];
        }
        if (pv) {
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] -= a2 * tp.v[w];
        }
        if (ppv) {
            const Pack<T> ppc = s_ppc[lane];
#pragma unroll
            for (int w = 0; w < W; ++w) res.v[w] -= ppc.v[w] * tpp.v[w];
        }
        st_pack(out + p * LPP, res);
        if (more) {
#pragma unroll
            for (int o = 0; o < 2 * R; ++o) win[o] = win[o + 1];
            win[2 * R] = nxt;
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_stencil_pass(const StencilOp& op, const Run& r, const StencilPass& p,
                                bool jacobi, cudaStream_t st)
{
    constexpr int W = 16 / sizeof(T);
    constexpr int LPP = CW / W;
    constexpr int TY = kThreads / LPP / TX;
    KArgs a;
    a.p = p;
    a.op = op;
    a.shift_of = r.shift_of;
    a.sigma = r.sigma;
    a.jac = r.jac;
    a.chunk_active = r.chunk_active;
    a.n = r.n;
    const int N = op.N;
    dim3 grid(((N + TX - 1) / TX) * ((N + TY - 1) / TY), (N + ZB - 1) / ZB, r.nchunk);
    if (op.order == 2) {
        if (jacobi) stencil_pass_kernel<T, 1, true><<<grid, kThreads, 0, st>>>(a);
        else stencil_pass_kernel<T, 1, false><<<grid, kThreads, 0, st>>>(a);
    } else {
        if (jacobi) stencil_pass_kernel<T, 2, true><<<grid, kThreads, 0, st>>>(a);
        else stencil_pass_kernel<T, 2, false><<<grid, kThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_stencil_pass<float>(const StencilOp&, const Run&, const StencilPass&,
                                                bool, cudaStream_t);
template cudaError_t launch_stencil_pass<double>(const StencilOp&, const Run&, const StencilPass&,
                                                 bool, cudaStream_t);

}  // namespace evc
