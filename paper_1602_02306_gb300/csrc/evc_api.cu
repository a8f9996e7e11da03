// evc_api.cu -- host side of libevc: the C ABI of include/evc.h.
//
// A call of evc_count_slices runs Algorithm 2 of the paper for S shifts and
// m probes at once: the S*m (shift, probe) columns are packed into 32-wide
// chunks, and every Lanczos step (Algorithm 1) is a fixed sequence of kernel
// launches over all active chunks:
//   operator passes  w = M (A - sigma I) M q_i - beta_i q_{i-1}
//   reorth           h = Q_i^T w, alpha_i = h_i, w -= Q_i h, ||w||^2
//   finish           beta_{i+1}, breakdown, eig(J_i) -> quadrature, stop rule
// The whole k-step sequence is captured once into a CUDA graph and replayed;
// the per-call values (shifts, seed, tol) live in device memory so a replay
// needs only a few small copies.  Shifts that meet the stop rule switch their
// chunks off on the device and the kernels skip them.
#include "evc_internal.cuh"
#include "../../include/evc.h"

#include <algorithm>
#include <complex>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace evc;

namespace {

enum { OP_CSR = 0, OP_STENCIL = 1 };

struct GraphKey {
    int S = -1, m = -1, kmax = -1, adaptive = -1, prec_version = -1, profile = -1, shared = -1,
        tinv = -1;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool operator==(const GraphKey& o) const
    {
        return S == o.S && m == o.m && kmax == o.kmax && adaptive == o.adaptive &&
               prec_version == o.prec_version && profile == o.profile && ws == o.ws &&
               ws_bytes == o.ws_bytes && shared == o.shared && tinv == o.tinv;
    }
};

}  // namespace

struct evc_ctx {
    int op = OP_CSR;
    int precision = EVC_FP64;
    size_t tsize = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n = 0;
    // CSR
    CsrOp csr{};
    int64_t nnz = 0;
    void* own_rowptr = nullptr;
    void* own_col = nullptr;
    void* own_val = nullptr;
    double* own_diag = nullptr;
    int32_t* own_perm = nullptr;
    // stencil
    StencilOp sten{};
    void* own_V = nullptr;
    int val_fp32 = 0;             // type of the values given at creation (1: float32)
    void* stage = nullptr;        // device staging of host values of the other type
    size_t stage_bytes = 0;
    // preconditioner
    int prec = EVC_PREC_IDENTITY;
    double jac_eps = 1e-3;
    int cheb_degree = 0;
    double cheb_c = 1.0;
    double cheb_a = 0, cheb_b = 0;
    std::vector<double> cheb_coef;
    // p_d in factored form (roots of p_d): conjugate pairs (re +- i im) and
    // real roots, empty when the factorisation failed its check
    struct ChebFactor { double re, im; bool pair; };
    std::vector<ChebFactor> cheb_fac;
    double cheb_g = 1.0, cheb_sign = 1.0;   // |leading coefficient|^(1/d), its sign
    int cheb_form = EVC_CHEB_FACTORED;
    int basis_bf16 = 0;
    int reorth_rows = 0;          // rows per block of the reorthogonalisation kernels (0: by n)
    // stencil operator segment of a step split into this many chunk groups on
    // concurrent streams (1: one stream); aux[g - 1] is the stream of group g
    int sten_groups = 1;
    cudaStream_t aux[kMaxStencilGroups - 1] = {};
    int method = EVC_METHOD_LANCZOS;
    int shared_krylov = 1;        // identity preconditioner: shifts share one run
    int tinv_lanczos = 0;         // Jacobi: the T^{-1}-inner-product process (Eq. lanT1)
    int prec_version = 0;
    int quad_rule = EVC_QUAD_GAUSS;
    int min_steps = 3;
    int64_t probe_offset = 0;
    // workspace
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    // pinned staging: per-call parameters (guarded by an event) and results
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
    void* pinres = nullptr;
    size_t pinres_bytes = 0;
    cudaEvent_t param_ev = nullptr;
    // launch list of the enqueued sequence (with timing events when profiling)
    bool profile = false;
    // bytes of a launch = fixed + per_chunk * (chunks active in that step);
    // span = 1: not a launch but the interval of a concurrent chunk-group
    // segment, whose launches carry no events of their own
    struct Rec { int kind, step; double fixed, per_chunk; cudaEvent_t e0, e1; int span; };
    std::vector<Rec> recs;
    bool in_span = false;         // enqueueing inside a chunk-group segment
    bool span_sum = false;        // ... the group whose launches the span record sums
    double span_frac = 1.0;       // share of the chunks in the current group
    double span_fixed = 0.0, span_per = 0.0;
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
    // graph
    bool use_graph = true;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    // last run
    Run run{};
    bool have_run = false;
    std::string err;
};

namespace {

int fail(evc_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(evc_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, EVC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Row blocks per chunk of the reorthogonalisation kernels.  It depends on n
// only, never on how many chunks share the launch, so the summation order of
// every dot product -- and therefore every result -- is the same whether a
// column runs alone or batched with others.  By default 3456 rows per block
// (54 tiles of the update kernel) keeps each block's bulk-copy pipeline long
// (the 64^3 Hamiltonian with four chunks gets 304 blocks, two per SM), and a
// problem with fewer than 64 x 3456 rows gets 64 blocks per chunk of at least
// 64 rows, so that small problems still spread over the GPU.
int default_reorth_rows(int64_t n)
{
    const int64_t r = (n + 63) / 64;
    return (int)std::min<int64_t>(3456, std::max<int64_t>(kMinReorthRows, r));
}

int choose_nblk(int64_t n, int rows)
{
    if (rows <= 0) rows = default_reorth_rows(n);
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + rows - 1) / rows, 65535));
}

struct Layout {
    size_t total;
    int nchunk, ncol, nblk;
};

bool uses_work(const evc_ctx* c) { return c->op == OP_STENCIL && c->prec == EVC_PREC_CHEB_KINETIC; }
bool uses_jac(const evc_ctx* c) { return c->prec == EVC_PREC_JACOBI; }
// T^{-1}-inner-product Lanczos (Eq. lanT1): with the Jacobi T = M^2 only; the
// identity preconditioner makes it Algorithm 1 itself.
bool uses_tinv(const evc_ctx* c)
{
    return c->tinv_lanczos && c->prec == EVC_PREC_JACOBI && c->method == EVC_METHOD_LANCZOS;
}
int pass_mode(const evc_ctx* c, const Run& r)
{
    if (!uses_jac(c)) return PM_NONE;
    return r.tinv ? PM_TLEFT : PM_JACOBI;
}
// Shared mode (see Run): without a preconditioner the Lanczos process on
// A - tau I is the one on A shifted by tau, so several shifts read one run.
bool use_shared(const evc_ctx* c, int S)
{
    return S > 1 && c->shared_krylov && c->prec == EVC_PREC_IDENTITY &&
           c->method == EVC_METHOD_LANCZOS;
}

// Carve the workspace into the run's arrays with one cursor, so the size
// query (base = 0) and the real carving can never disagree.  Every array
// starts on a 256-byte boundary.
size_t carve(const evc_ctx* c, int S, int m, int kmax, char* base, Run& r, void** work)
{
    const bool shared = use_shared(c, S);
    const int Sop = shared ? 1 : S;
    const int ncol_real = shared ? m : S * m;
    const int nchunk = (ncol_real + CW - 1) / CW;
    const int ncol = nchunk * CW;
    const int nblk = choose_nblk(c->n, c->reorth_rows);
    const int nblk_max = reorth_max_blocks(c->n);   // any allowed value fits
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t vec = (size_t)c->n * CW * c->tsize;
    r.n = c->n;
    r.S = S;
    r.m = m;
    r.kmax = kmax;
    r.ncol = ncol;
    r.ncol_real = ncol_real;
    r.shared = shared ? 1 : 0;
    r.nq = S * m;
    r.Sop = Sop;
    r.nchunk = nchunk;
    r.nblk = nblk;
    r.slot_stride = c->n * CW;
    r.chunk_stride = (int64_t)(kmax + 1) * c->n * CW;
    r.basis = take((size_t)nchunk * (kmax + 1) * vec);
    void* w = uses_work(c) ? take(3 * (size_t)nchunk * vec) : nullptr;
    if (work) *work = w;
    r.jac = uses_jac(c) ? take((size_t)Sop * c->n * c->tsize) : nullptr;
    r.dsh = c->op == OP_CSR ? take((size_t)Sop * c->n * c->tsize) : nullptr;
    r.tinv = uses_tinv(c) ? 1 : 0;
    r.tinvd = r.tinv ? take((size_t)Sop * c->n * c->tsize) : nullptr;
    auto D = [&](size_t cnt) { return reinterpret_cast<double*>(take(cnt * 8)); };
    auto I = [&](size_t cnt) { return reinterpret_cast<int*>(take(cnt * 4)); };
    r.sigma = D(ncol);
    r.alpha = D((size_t)kmax * ncol);
    r.beta = D((size_t)(kmax + 1) * ncol);
    r.scl = D((size_t)(kmax + 1) * ncol);
    r.g = D((size_t)kmax * ncol);
    r.ppc = D(ncol);
    r.colscale = D(ncol);
    r.quad = D((size_t)S * m);
    r.quad_final = D((size_t)S * m);
    r.probe_id = reinterpret_cast<int64_t*>(take((size_t)ncol * 8));
    r.shift_of = I(ncol);
    r.kdone = I(ncol);
    r.shifts = D(S);
    r.Lprev = D(S);
    r.Lprev2 = D(S);
    r.Lfinal = D(S);
    r.steps = I(S);
    r.sdone = I(S);
    r.stol = D(S);
    r.skmax = I(S);
    r.opshift = D(Sop);
    r.chunk_active = I(nchunk);
    r.cnt_upd = I(nchunk);
    r.nactive = I(kmax + 1);
    r.part_dot = D((size_t)nchunk * nblk_max * kmax * CW);
    r.part_gram = D((size_t)nchunk * nblk_max * kmax * CW);
    r.hbuf = D((size_t)kmax * ncol);
    r.gram = D((size_t)kmax * (kmax + 1) / 2 * ncol);
    r.part_nrm = D((size_t)nchunk * nblk_max * CW);
    r.err = I(1);
    r.seed = reinterpret_cast<uint64_t*>(take(8));
    r.breakdown_rel = c->precision == EVC_FP64 ? 1e-12 : 1e-6;
    r.ga = c->quad_rule == EVC_QUAD_GA ? 1 : 0;
    r.min_steps = c->min_steps;
    r.basis_bf16 = c->basis_bf16;
    r.arnoldi = c->method == EVC_METHOD_ARNOLDI ? 1 : 0;
    r.hess = r.arnoldi ? D((size_t)kmax * (kmax + 1) / 2 * ncol) : nullptr;
    return off;
}

Layout layout(const evc_ctx* c, int S, int m, int kmax)
{
    Run r{};
    Layout L;
    L.total = carve(c, S, m, kmax, nullptr, r, nullptr);
    L.nchunk = r.nchunk;
    L.ncol = r.ncol;
    L.nblk = r.nblk;
    return L;
}

// ------------------------------------------------------------ conversions

template <typename D, typename S_>
__global__ void convert_kernel(D* dst, const S_* src, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}

__global__ void csr_diag_kernel(const int64_t* rp, const int32_t* col, const void* val, int fp32,
                                double* diag, int64_t n)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
            if (col[k] == r)
                d += fp32 ? (double)static_cast<const float*>(val)[k]
                          : static_cast<const double*>(val)[k];
        diag[r] = d;
    }
}

// Free the staging buffer of upload_values (after the stream has used it).
int release_stage(evc_ctx* ctx)
{
    if (!ctx->stage) return EVC_OK;
    CU(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    return EVC_OK;
}

// Copy `count` matrix values (float32 when src_fp32, else float64; host or
// device) into dst in the context's type.  With diag set (CSR contexts), also
// form the FP64 diagonal from the values as given, before any rounding to the
// context's type: the Jacobi scaling and the shifted diagonal derive from it.
int upload_values(evc_ctx* ctx, void* dst, const void* src, int64_t count, int src_fp32,
                  int on_device, double* diag = nullptr)
{
    const size_t ssz = src_fp32 ? 4 : 8;
    const bool same = (src_fp32 ? 4u : 8u) == ctx->tsize;
    const int dblocks = (int)std::min<int64_t>((ctx->n + 255) / 256, 152 * 16);
    auto form_diag = [&](const void* vals) -> int {
        if (!diag) return EVC_OK;
        csr_diag_kernel<<<dblocks, 256, 0, ctx->stream>>>(ctx->csr.row_ptr, ctx->csr.col, vals,
                                                          src_fp32, diag, ctx->n);
        CU(cudaGetLastError());
        return EVC_OK;
    };
    if (same) {
        CU(cudaMemcpyAsync(dst, src, count * ssz, on_device ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyHostToDevice,
                           ctx->stream));
        return form_diag(dst);
    }
    const void* dsrc = src;
    if (!on_device) {
        // host values of the other type pass through a device staging buffer
        // the context keeps (grown on demand), so repeated updates allocate nothing
        const size_t need = (size_t)count * ssz;
        if (ctx->stage_bytes < need) {
            CU(cudaStreamSynchronize(ctx->stream));
            if (ctx->stage) cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
            CU(cudaMalloc(&ctx->stage, need));
            ctx->stage_bytes = need;
        }
        CU(cudaMemcpyAsync(ctx->stage, src, need, cudaMemcpyHostToDevice, ctx->stream));
        dsrc = ctx->stage;
    }
    int rc = form_diag(dsrc);
    if (rc) return rc;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
    if (ctx->tsize == 4)
        convert_kernel<float, double><<<blocks, 256, 0, ctx->stream>>>(
            static_cast<float*>(dst), static_cast<const double*>(dsrc), count);
    else
        convert_kernel<double, float><<<blocks, 256, 0, ctx->stream>>>(
            static_cast<double*>(dst), static_cast<const float*>(dsrc), count);
    CU(cudaGetLastError());
    return EVC_OK;
}

// ---------------------------------------------------------- Chebyshev M

// Symbol of -1/2 d^2/dx^2 (one axis) at wavenumber theta.
double axis_symbol(int order, double h, double th)
{
    if (order == 2) return (1.0 - std::cos(th)) / (h * h);
    return (30.0 - 32.0 * std::cos(th) + 2.0 * std::cos(2.0 * th)) / (24.0 * h * h);
}

double cheb_eval(const std::vector<double>& c, double a, double b, double x)
{
    // Clenshaw summation of sum_j c_j T_j(t), t = (2x - a - b)/(b - a)
    const double t = (2.0 * x - a - b) / (b - a);
    double b1 = 0.0, b2 = 0.0;
    for (int j = (int)c.size() - 1; j >= 1; --j) {
        const double b0 = c[j] + 2.0 * t * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return c[0] + t * b1 - b2;
}

// p(t) = sum_j c_j T_j(t) and p'(t) for complex t (Clenshaw summation; dc are
// the Chebyshev coefficients of p').
void cheb_val_der(const std::vector<double>& c, const std::vector<double>& dc,
                  std::complex<double> t, std::complex<double>& p, std::complex<double>& dp)
{
    auto clen = [&](const std::vector<double>& cc) {
        std::complex<double> b1 = 0.0, b2 = 0.0;
        for (int j = (int)cc.size() - 1; j >= 1; --j) {
            const std::complex<double> b0 = cc[j] + 2.0 * t * b1 - b2;
            b2 = b1;
            b1 = b0;
        }
        return cc.empty() ? std::complex<double>(0.0) : cc[0] + t * b1 - b2;
    };
    p = clen(c);
    dp = clen(dc);
}

// Roots of p_d (Aberth-Ehrlich simultaneous iteration on the Chebyshev series
// in t = (2x - a - b)/(b - a)), mapped to x and sorted into conjugate pairs
// (ascending real part) followed by real roots.  The factored product
//   sign * prod_pairs g^2 ((x - re)^2 + im^2) * prod_reals g (x - r)
// must reproduce p_d on [a, b] to 1e-9 relative, else false.
bool cheb_factor(const std::vector<double>& c, double a, double b,
                 std::vector<evc_ctx::ChebFactor>& fac, double& g, double& sgn)
{
    typedef std::complex<double> cd;
    const int d = (int)c.size() - 1;
    fac.clear();
    if (d < 1 || c[d] == 0.0) return false;
    std::vector<double> tmp(d + 2, 0.0);
    for (int k = d; k >= 1; --k) tmp[k - 1] = tmp[k + 1] + 2.0 * k * c[k];
    tmp[0] *= 0.5;
    std::vector<double> dc(tmp.begin(), tmp.begin() + d);
    std::vector<cd> z(d);
    const double pi = 3.141592653589793238462643;
    for (int k = 0; k < d; ++k) z[k] = std::polar(1.3, 2.0 * pi * k / d + 0.4);
    for (int it = 0; it < 2000; ++it) {
        double mx = 0.0;
        for (int k = 0; k < d; ++k) {
            cd p, dp;
            cheb_val_der(c, dc, z[k], p, dp);
            if (std::abs(p) == 0.0) continue;
            const cd ratio = p / dp;
            cd sum = 0.0;
            for (int j = 0; j < d; ++j)
                if (j != k) sum += 1.0 / (z[k] - z[j]);
            const cd w = ratio / (1.0 - ratio * sum);
            if (!std::isfinite(w.real()) || !std::isfinite(w.imag())) return false;
            z[k] -= w;
            mx = std::max(mx, std::abs(w) / (1.0 + std::abs(z[k])));
        }
        if (mx < 1e-15) break;
    }
    std::vector<cd> x(d);
    for (int k = 0; k < d; ++k) x[k] = 0.5 * (b - a) * z[k] + 0.5 * (a + b);
    std::vector<bool> used(d, false);
    std::vector<evc_ctx::ChebFactor> pairs, reals;
    for (int k = 0; k < d; ++k) {
        if (used[k]) continue;
        if (std::abs(x[k].imag()) <= 1e-9 * (1.0 + std::abs(x[k]))) {
            used[k] = true;
            reals.push_back({x[k].real(), 0.0, false});
            continue;
        }
        int best = -1;
        double bd = 1e300;
        for (int j = 0; j < d; ++j) {
            if (j == k || used[j]) continue;
            const double dist = std::abs(x[j] - std::conj(x[k]));
            if (dist < bd) {
                bd = dist;
                best = j;
            }
        }
        if (best < 0 || bd > 1e-7 * (1.0 + std::abs(x[k]))) return false;
        used[k] = used[best] = true;
        pairs.push_back({0.5 * (x[k].real() + x[best].real()), std::abs(x[k].imag()), true});
    }
    auto by_re = [](const evc_ctx::ChebFactor& u, const evc_ctx::ChebFactor& v) { return u.re < v.re; };
    std::sort(pairs.begin(), pairs.end(), by_re);
    std::sort(reals.begin(), reals.end(), by_re);
    fac = pairs;
    fac.insert(fac.end(), reals.begin(), reals.end());
    const double lead = c[d] * std::ldexp(1.0, d - 1) * std::pow(2.0 / (b - a), d);
    g = std::pow(std::fabs(lead), 1.0 / d);
    sgn = lead < 0 ? -1.0 : 1.0;
    for (int m = 0; m <= 4000; ++m) {
        const double xx = a + (b - a) * m / 4000.0;
        double prod = sgn;
        for (const auto& f : fac)
            prod *= f.pair ? g * g * ((xx - f.re) * (xx - f.re) + f.im * f.im) : g * (xx - f.re);
        const double ref = cheb_eval(c, a, b, xx);
        if (!(std::fabs(prod - ref) <= 1e-9 * std::max(std::fabs(ref), 1e-300))) {
            fac.clear();
            return false;
        }
    }
    return true;
}

}  // namespace

int evc::cheb_coefficients(int degree, double a, double b, double* coef)
{
    // Interpolation of f(x) = x^(-1/2) at the d+1 Chebyshev points of the first
    // kind mapped to [a, b]: c_j = (2/(d+1)) sum_k f(x_k) T_j(t_k), c_0 halved.
    const int np = degree + 1;
    const double pi = 3.141592653589793238462643;
    std::vector<double> f(np);
    for (int k = 0; k < np; ++k) {
        const double th = pi * (2 * k + 1) / (2.0 * np);
        f[k] = 1.0 / std::sqrt(0.5 * (a + b) + 0.5 * (b - a) * std::cos(th));
    }
    for (int j = 0; j <= degree; ++j) {
        double s = 0.0;
        for (int k = 0; k < np; ++k) s += f[k] * std::cos(j * pi * (2 * k + 1) / (2.0 * np));
        coef[j] = (j == 0 ? 1.0 : 2.0) * s / np;
    }
    return 0;
}

namespace {

// The kinetic Chebyshev preconditioner M = p_d(K) of a periodic stencil of
// this order and spacing, K = -1/2 Lap_h + cI: its interval [a, b] (the
// closed-form bounds of spec(K)), coefficients, the smallest value of p_d on
// the exact discrete spectrum of an N^3 grid (N = 0: not checked), and the
// factored form (empty when the factorisation fails its check).
struct ChebSetup {
    double a = 0, b = 0, pmin = 0, g = 1, sign = 1;
    std::vector<double> coef;
    std::vector<evc_ctx::ChebFactor> fac;
};

const char* cheb_setup(int order, double h, int d, double c, int N, ChebSetup& out)
{
    if (order != 2 && order != 4) return "stencil order must be 2 or 4";
    if (!(h > 0.0) || !std::isfinite(h)) return "grid spacing must be > 0";
    if (d < 1 || d > 32) return "Chebyshev degree must be an integer in [1, 32]";
    if (!(c > 0.0) || !std::isfinite(c)) return "kinetic shift c must be > 0";
    out.a = c;
    out.b = c + (order == 2 ? 6.0 : 8.0) / (h * h);
    out.coef.assign(d + 1, 0.0);
    evc::cheb_coefficients(d, out.a, out.b, out.coef.data());
    // T = M^2 is SPD iff p_d > 0 on the spectrum of K: the periodic
    // stencil's eigenvalues are c + sum over axes of the axis symbol at
    // theta = 2 pi k / N.
    out.pmin = 1e300;
    if (N > 0) {
        std::vector<double> sym(N);
        for (int k = 0; k < N; ++k) sym[k] = axis_symbol(order, h, 2.0 * M_PI * k / N);
        std::sort(sym.begin(), sym.end());
        sym.erase(std::unique(sym.begin(), sym.end()), sym.end());
        for (size_t i1 = 0; i1 < sym.size(); ++i1)
            for (size_t i2 = i1; i2 < sym.size(); ++i2)
                for (size_t i3 = i2; i3 < sym.size(); ++i3)
                    out.pmin = std::min(out.pmin, cheb_eval(out.coef, out.a, out.b,
                                                            out.a + sym[i1] + sym[i2] + sym[i3]));
    }
    if (!cheb_factor(out.coef, out.a, out.b, out.fac, out.g, out.sign)) out.fac.clear();
    return nullptr;
}

}  // namespace

namespace {

// ------------------------------------------------------- step sequence

cudaEvent_t pool_event(evc_ctx* ctx)
{
    if (ctx->evnext == ctx->evpool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->evpool.push_back(e);
    }
    return ctx->evpool[ctx->evnext++];
}

// Enqueue one kernel launch, bracketed by timing events when profiling.
template <class F>
int rec(evc_ctx* ctx, int kind, int step, double fixed, double per_chunk, F&& launch)
{
    evc_ctx::Rec r{kind, step, fixed, per_chunk, nullptr, nullptr, 0};
    if (ctx->in_span) {
        // concurrent with the other groups: timed as one span, bytes summed
        // once over the whole chunk range
        if (ctx->span_sum) {
            ctx->span_fixed += fixed;
            ctx->span_per += per_chunk;
        }
        r.fixed = fixed * ctx->span_frac;
        r.per_chunk = per_chunk * ctx->span_frac;
    } else if (ctx->profile) {
        r.e0 = pool_event(ctx);
        r.e1 = pool_event(ctx);
        if (!r.e0 || !r.e1) return fail(ctx, EVC_ECUDA, "cudaEventCreate failed");
        // external record nodes when captured, so the events can be timed after a replay
        CU(cudaEventRecordWithFlags(r.e0, ctx->stream, cudaEventRecordExternal));
    }
    cudaError_t e = launch();
    if (e != cudaSuccess)
        return fail(ctx, EVC_ECUDA, "kernel launch (class %d, step %d): %s", kind, step,
                    cudaGetErrorString(e));
    if (r.e1) CU(cudaEventRecordWithFlags(r.e1, ctx->stream, cudaEventRecordExternal));
    ctx->recs.push_back(r);
    return EVC_OK;
}

// Enqueue body() -- the stencil launches of one operator application -- once
// per chunk group, each group on its own stream, forked from and joined back
// into the context's stream.  The chunks of a step are independent until the
// reorthogonalisation, so the groups' launches overlap and the tail wave of
// one group's pass runs beside the next pass of another instead of leaving
// SMs idle.  Every chunk is computed by the same kernels as without groups,
// so results are bitwise the same.  When profiling, the segment is one span
// record (kind `kind`) timed on the context's stream.
template <class F>
int grouped(evc_ctx* ctx, const Run& r, int kind, int step, F&& body)
{
    const int G = std::min(ctx->sten_groups, r.nchunk);
    if (G <= 1 || ctx->in_span) return body();
    cudaStream_t s0 = ctx->stream;
    for (int g = 1; g < G; ++g)
        if (!ctx->aux[g - 1]) CU(cudaStreamCreateWithFlags(&ctx->aux[g - 1], cudaStreamNonBlocking));
    cudaEvent_t fork = pool_event(ctx);
    if (!fork) return fail(ctx, EVC_ECUDA, "cudaEventCreate failed");
    evc_ctx::Rec span{kind, step, 0.0, 0.0, nullptr, nullptr, 1};
    if (ctx->profile) {
        span.e0 = pool_event(ctx);
        span.e1 = pool_event(ctx);
        if (!span.e0 || !span.e1) return fail(ctx, EVC_ECUDA, "cudaEventCreate failed");
        CU(cudaEventRecordWithFlags(span.e0, s0, cudaEventRecordExternal));
    }
    CU(cudaEventRecord(fork, s0));
    ctx->in_span = true;
    ctx->span_fixed = ctx->span_per = 0.0;
    int rc = EVC_OK;
    for (int g = 0; g < G && !rc; ++g) {
        const int c0 = (int)((int64_t)r.nchunk * g / G), c1 = (int)((int64_t)r.nchunk * (g + 1) / G);
        cudaStream_t sg = g == 0 ? s0 : ctx->aux[g - 1];
        if (g > 0) {
            cudaError_t e = cudaStreamWaitEvent(sg, fork, 0);
            if (e != cudaSuccess) {
                rc = fail(ctx, EVC_ECUDA, "stream fork: %s", cudaGetErrorString(e));
                break;
            }
        }
        ctx->stream = sg;
        ctx->sten.c0 = c0;
        ctx->sten.cn = c1 - c0;
        ctx->span_sum = g == 0;
        ctx->span_frac = (double)(c1 - c0) / r.nchunk;
        rc = body();
        if (g > 0) {
            // join: the context's stream waits for this group (also after an
            // error, so that a capture ends with every stream joined)
            cudaEvent_t join = pool_event(ctx);
            cudaError_t e = join ? cudaEventRecord(join, sg) : cudaErrorMemoryAllocation;
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, join, 0);
            if (e != cudaSuccess && !rc) rc = fail(ctx, EVC_ECUDA, "stream join: %s", cudaGetErrorString(e));
        }
    }
    ctx->stream = s0;
    ctx->sten.c0 = ctx->sten.cn = 0;
    ctx->in_span = ctx->span_sum = false;
    ctx->span_frac = 1.0;
    if (rc) return rc;
    span.fixed = ctx->span_fixed;
    span.per_chunk = ctx->span_per;
    if (span.e1) CU(cudaEventRecordWithFlags(span.e1, s0, cudaEventRecordExternal));
    if (ctx->profile) ctx->recs.push_back(span);
    return EVC_OK;
}

enum BKind { B_ZERO, B_XMUL, B_BUF };
struct BTerm {
    BKind kind = B_ZERO;
    double gamma = 0.0;
    void* buf = nullptr;
};

template <typename T>
int stencil(evc_ctx* ctx, const Run& r, int step, const StencilPass& p, int pmode)
{
    // compulsory traffic: the stencil operand and every pointwise operand read
    // once, the output written once (per active chunk); V and Jacobi scales once
    const double vchunk = (double)r.n * CW * sizeof(T);
    const double per = vchunk * (2 + (p.x ? 1 : 0) + (p.prev ? 1 : 0) + (p.pp ? 1 : 0));
    double fixed = p.useV ? (double)r.n * sizeof(T) : 0.0;
    if (pmode != PM_NONE) fixed += (double)r.Sop * r.n * sizeof(T);
    return rec(ctx, EVC_K_STENCIL, step, fixed, per,
               [&] { return launch_stencil_pass<T>(ctx->sten, r, p, pmode, ctx->stream); });
}

// y = p_d(K) x by Clenshaw's recurrence b_j = c_j x + 2 K~ b_{j+1} - b_{j+2},
// y = c_0 x + K~ b_1 - b_2, K~ = (2K - (a+b)I)/(b-a).  Terms that are still
// multiples of x are folded into the next pass, so degree d costs d passes;
// b_j overwrites b_{j+2} in place (it is read only at its own point).
// y = p_d(K) x in factored form: for each conjugate pair of roots of p_d,
//   u = g (K - re) x,   x <- g (K - re) u + g^2 im^2 x
// (two passes that move 5 vectors per degree 2, against 8 for two Clenshaw
// steps), then one pass g (K - r) per real root; the sign of the leading
// coefficient and the "- beta_i q_{i-1}" term ride on the last pass.  The
// shifted quadratic form has no cancellation; the factorisation is checked
// against the series when the preconditioner is set.  Wa is scratch; the
// running product lives in Wb (updated in place: a pass reads its x operand
// only at its own point).
template <typename T>
int enqueue_cheb_factored(evc_ctx* ctx, const Run& r, int step, const void* x, int64_t x_cs,
                          const double* xscale, void* Wa, void* Wb, void* out, int64_t out_cs,
                          const void* pp, int64_t pp_cs, const double* ppc)
{
    const int64_t wcs = r.n * CW;
    const double g = ctx->cheb_g, c = ctx->cheb_c;
    const void* cur = x;
    int64_t cur_cs = x_cs;
    const double* cur_sc = xscale;
    const size_t nf = ctx->cheb_fac.size();
    for (size_t f = 0; f < nf; ++f) {
        const evc_ctx::ChebFactor& F = ctx->cheb_fac[f];
        const bool last = f + 1 == nf;
        const double sg = last ? ctx->cheb_sign : 1.0;
        void* dst = last ? out : Wb;
        const int64_t dst_cs = last ? out_cs : wcs;
        StencilPass p{};
        if (F.pair) {
            StencilPass pa{};
            pa.in = cur;
            pa.in_cs = cur_cs;
            pa.insc = cur_sc;
            pa.k1 = g;
            pa.k0 = g * (c - F.re);
            pa.out = Wa;
            pa.out_cs = wcs;
            int rc = stencil<T>(ctx, r, step, pa, PM_NONE);
            if (rc) return rc;
            p.in = Wa;
            p.in_cs = wcs;
            p.k1 = sg * g;
            p.k0 = sg * g * (c - F.re);
            p.x = cur;
            p.x_cs = cur_cs;
            p.xs = cur_sc;
            p.a0 = sg * g * g * F.im * F.im;
        } else {
            // reads cur with its halo: never in place
            if (!last && cur == Wb) dst = Wa;
            p.in = cur;
            p.in_cs = cur_cs;
            p.insc = cur_sc;
            p.k1 = sg * g;
            p.k0 = sg * g * (c - F.re);
        }
        p.out = dst;
        p.out_cs = dst_cs;
        if (last) {
            p.pp = pp;
            p.pp_cs = pp_cs;
            p.ppc = pp ? ppc : nullptr;
        }
        int rc = stencil<T>(ctx, r, step, p, PM_NONE);
        if (rc) return rc;
        cur = dst;
        cur_cs = dst_cs;
        cur_sc = nullptr;
    }
    return EVC_OK;
}

template <typename T>
int enqueue_cheb(evc_ctx* ctx, const Run& r, int step, const void* x, int64_t x_cs,
                 const double* xscale, void* W0, void* W1, void* out, int64_t out_cs,
                 const void* pp, int64_t pp_cs, const double* ppc)
{
    if (ctx->cheb_form == EVC_CHEB_FACTORED && !ctx->cheb_fac.empty())
        return enqueue_cheb_factored<T>(ctx, r, step, x, x_cs, xscale, W0, W1, out, out_cs, pp,
                                        pp_cs, ppc);
    const int d = ctx->cheb_degree;
    const std::vector<double>& c = ctx->cheb_coef;
    const double a = ctx->cheb_a, b = ctx->cheb_b;
    const double kap1 = 2.0 / (b - a), kap0 = (2.0 * ctx->cheb_c - a - b) / (b - a);
    const int64_t wcs = r.n * CW;
    BTerm b1, b2;   // b_{j+1}, b_{j+2}
    for (int j = d; j >= 0; --j) {
        const bool final_ = (j == 0);
        const double f = final_ ? 1.0 : 2.0;
        if (!final_ && b1.kind == B_ZERO && b2.kind == B_ZERO) {
            b1.kind = B_XMUL;
            b1.gamma = c[j];
            continue;
        }
        StencilPass p{};
        if (b1.kind == B_XMUL) {
            p.in = x;
            p.in_cs = x_cs;
            p.insc = xscale;
            p.k1 = f * b1.gamma * kap1;
            p.k0 = f * b1.gamma * kap0 + c[j];
            if (b2.kind == B_XMUL) p.k0 -= b2.gamma;
        } else {
            p.in = b1.buf;
            p.in_cs = wcs;
            p.k1 = f * kap1;
            p.k0 = f * kap0;
            p.x = x;
            p.x_cs = x_cs;
            p.xs = xscale;
            p.a0 = c[j];
            if (b2.kind == B_XMUL) p.a0 -= b2.gamma;
            if (b2.kind == B_BUF) {
                p.prev = b2.buf;
                p.prev_cs = wcs;
                p.a2 = 1.0;
            }
        }
        void* dst;
        int64_t dst_cs = wcs;
        if (final_) {
            dst = out;
            dst_cs = out_cs;
            p.pp = pp;
            p.pp_cs = pp_cs;
            p.ppc = pp ? ppc : nullptr;
        } else if (b2.kind == B_BUF) {
            dst = b2.buf;
        } else {
            dst = (b1.kind == B_BUF && b1.buf == W0) ? W1 : W0;
        }
        p.out = dst;
        p.out_cs = dst_cs;
        int rc = stencil<T>(ctx, r, step, p, PM_NONE);
        if (rc) return rc;
        if (final_) break;
        BTerm nb;
        nb.kind = B_BUF;
        nb.buf = dst;
        b2 = b1;
        b1 = nb;
    }
    return EVC_OK;
}

// Arnoldi (Sec. 4, Algorithm 3): w = T (A - sigma I) q_i into slot i, with T
// used without its factorisation and no three-term term.  Chebyshev:
// T = p_d(K)^2, i.e. (H - sigma I) into slot i, M into W2, M back into slot i;
// Jacobi: T = diag(m^2) as a row scaling after the plain operator pass.
template <typename T>
int enqueue_arnoldi_operator(evc_ctx* ctx, const Run& r, int i, void* work)
{
    cudaStream_t st = ctx->stream;
    const double vchunk = (double)r.n * CW * sizeof(T);
    T* basis = static_cast<T*>(r.basis);
    T* qi = basis + (int64_t)(i - 1) * r.slot_stride;
    T* wout = basis + (int64_t)i * r.slot_stride;
    const double* si = r.scl + (int64_t)(i - 1) * r.ncol;
    const int64_t vstride = r.n * CW;
    int rc;
    if (ctx->op == OP_CSR) {
        const double fixed = (double)ctx->nnz * (sizeof(T) + 4) + 8.0 * (r.n + 1) +
                             (double)r.Sop * r.n * sizeof(T);
        const double per = (double)ctx->nnz * CW * sizeof(T) + vchunk;
        rc = rec(ctx, EVC_K_CSR, i, fixed, per,
                 [&] { return launch_csr_pass<T>(ctx->csr, r, i, PM_NONE, st); });
    } else {
        StencilPass p{};
        p.in = qi;
        p.in_cs = r.chunk_stride;
        p.insc = si;
        p.k1 = 1.0;
        p.useV = 1;
        p.useSigma = 1;
        p.out = wout;
        p.out_cs = r.chunk_stride;
        rc = grouped(ctx, r, EVC_K_STENCIL, i, [&]() -> int {
            int rc2 = stencil<T>(ctx, r, i, p, PM_NONE);
            if (!rc2 && ctx->prec == EVC_PREC_CHEB_KINETIC) {
                T* W0 = static_cast<T*>(work);
                T* W1 = W0 + (int64_t)r.nchunk * vstride;
                T* W2 = W1 + (int64_t)r.nchunk * vstride;
                rc2 = enqueue_cheb<T>(ctx, r, i, wout, r.chunk_stride, nullptr, W0, W1, W2,
                                      vstride, nullptr, 0, nullptr);
                if (!rc2)
                    rc2 = enqueue_cheb<T>(ctx, r, i, W2, vstride, nullptr, W0, W1, wout,
                                          r.chunk_stride, nullptr, 0, nullptr);
            }
            return rc2;
        });
    }
    if (!rc && uses_jac(ctx))
        rc = rec(ctx, EVC_K_JACOBI, i, (double)r.Sop * r.n * sizeof(T), 2.0 * vchunk,
                 [&] { return launch_row_scale<T>(r, wout, r.chunk_stride, st); });
    return rc;
}

template <typename T>
int enqueue_all(evc_ctx* ctx, const Run& r, void* work, bool adaptive)
{
    cudaStream_t st = ctx->stream;
    const double vchunk = (double)r.n * CW * sizeof(T);
    const double colb = (double)r.ncol * 8;
    int rc = rec(ctx, EVC_K_INIT, 0, colb * 8, 0.0, [&] { return launch_init_state(r, st); });
    if (!rc && (uses_jac(ctx) || ctx->op == OP_CSR)) {
        // Jacobi scales and (CSR) the shifted operator's diagonal, per shift
        const double vdiag = ctx->op == OP_STENCIL ? ctx->sten.cd : 0.0;
        const double outs = (r.jac ? 1.0 : 0.0) + (r.dsh ? 1.0 : 0.0) + (r.tinvd ? 1.0 : 0.0);
        rc = rec(ctx, EVC_K_JACOBI, 0, outs * r.Sop * r.n * sizeof(T) + r.n * 8.0, 0.0, [&] {
            return launch_jacobi_scales<T>(r, ctx->op == OP_CSR ? ctx->csr.diag : nullptr,
                                           ctx->op == OP_STENCIL ? ctx->sten.V : nullptr, vdiag,
                                           ctx->jac_eps, r.arnoldi ? PM_NONE : pass_mode(ctx, r),
                                           st);
        });
    }
    // the probe (T^{-1} mode: y_1 = M q_1, after the scales)
    if (!rc)
        rc = rec(ctx, EVC_K_INIT, 0, r.tinv ? (double)r.Sop * r.n * sizeof(T) : 0.0, vchunk,
                 [&] { return launch_init_probe<T>(r, st); });
    if (rc) return rc;
    T* basis = static_cast<T*>(r.basis);
    const int64_t vstride = r.n * CW;
    for (int i = 1; i <= r.kmax && !rc; ++i) {
        T* qi = basis + (int64_t)(i - 1) * r.slot_stride;
        T* qprev = i >= 2 ? basis + (int64_t)(i - 2) * r.slot_stride : nullptr;
        T* wout = basis + (int64_t)i * r.slot_stride;
        const double* si = r.scl + (int64_t)(i - 1) * r.ncol;
        if (r.arnoldi) {
            rc = enqueue_arnoldi_operator<T>(ctx, r, i, work);
        } else if (ctx->op == OP_CSR) {
            // the CSR structure and values once; per chunk, one gathered 32-column
            // x row per stored entry, the output and q_{i-1}
            const int pm = pass_mode(ctx, r);
            const double fixed = (double)ctx->nnz * (sizeof(T) + 4) + 8.0 * (r.n + 1) +
                                 (pm != PM_NONE ? 2.0 : 1.0) * r.Sop * r.n * sizeof(T);
            const double per = (double)ctx->nnz * CW * sizeof(T) + vchunk * (1 + (qprev ? 1 : 0));
            rc = rec(ctx, EVC_K_CSR, i, fixed, per,
                     [&] { return launch_csr_pass<T>(ctx->csr, r, i, pm, st); });
        } else if (ctx->prec == EVC_PREC_CHEB_KINETIC) {
            T* W0 = static_cast<T*>(work);
            T* W1 = W0 + (int64_t)r.nchunk * vstride;
            T* W2 = W1 + (int64_t)r.nchunk * vstride;
            rc = grouped(ctx, r, EVC_K_STENCIL, i, [&]() -> int {
                // u = M q_i into W2
                int rc2 = enqueue_cheb<T>(ctx, r, i, qi, r.chunk_stride, si, W0, W1, W2, vstride,
                                          nullptr, 0, nullptr);
                if (rc2) return rc2;
                // t = (H - sigma I) u into W0
                StencilPass p{};
                p.in = W2;
                p.in_cs = vstride;
                p.k1 = 1.0;
                p.useV = 1;
                p.useSigma = 1;
                p.out = W0;
                p.out_cs = vstride;
                rc2 = stencil<T>(ctx, r, i, p, PM_NONE);
                if (rc2) return rc2;
                // w = M t - beta_i q_{i-1} into slot i
                return enqueue_cheb<T>(ctx, r, i, W0, vstride, nullptr, W1, W2, wout,
                                       r.chunk_stride, qprev, r.chunk_stride, r.ppc);
            });
        } else {
            StencilPass p{};
            p.in = qi;
            p.in_cs = r.chunk_stride;
            p.insc = si;
            p.k1 = 1.0;
            p.useV = 1;
            p.useSigma = 1;
            p.out = wout;
            p.out_cs = r.chunk_stride;
            p.pp = qprev;
            p.pp_cs = r.chunk_stride;
            p.ppc = qprev ? r.ppc : nullptr;
            rc = grouped(ctx, r, EVC_K_STENCIL, i,
                         [&]() -> int { return stencil<T>(ctx, r, i, p, pass_mode(ctx, r)); });
        }
        if (rc) return rc;
        // T^{-1} mode: the weights T^{-1} once per chunk and kernel
        const double tw = r.tinv ? vchunk / CW : 0.0;
        rc = rec(ctx, EVC_K_DOTS, i, 0.0, vchunk * (i + 1) + tw,
                 [&] { return launch_dots<T>(r, i, st); });
        if (!rc)
            rc = rec(ctx, EVC_K_REDUCE, i, colb * 3 * i, 2.0 * r.nblk * i * CW * 8,
                     [&] { return launch_reduce(r, i, st); });
        if (!rc)
            rc = rec(ctx, EVC_K_REDUCE, i, colb * (2.0 * i + i * (i + 1) / 2), 0.0,
                     [&] { return launch_coef(r, i, st); });
        if (!rc)
            rc = rec(ctx, EVC_K_UPDATE, i, 0.0, vchunk * (i + 2) + tw,
                     [&] { return launch_update<T>(r, i, st); });
        const bool last = (i == r.kmax);
        if (!rc && (adaptive || last))
            rc = rec(ctx, EVC_K_FINISH, i, colb * (2.0 * i + 2), 0.0,
                     [&] { return launch_finish(r, i, st); });
        if (!rc && adaptive)
            rc = rec(ctx, EVC_K_FINISH, i, colb, 0.0, [&] { return launch_active(r, i, st); });
    }
    return rc;
}

int ensure_pinned(evc_ctx* ctx, void** buf, size_t* have, size_t bytes)
{
    if (*have >= bytes) return EVC_OK;
    if (*buf) {
        CU(cudaStreamSynchronize(ctx->stream));
        cudaFreeHost(*buf);
    }
    *buf = nullptr;
    *have = 0;
    CU(cudaHostAlloc(buf, bytes, cudaHostAllocDefault));
    *have = bytes;
    return EVC_OK;
}

void drop_graph(evc_ctx* ctx)
{
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gkey = GraphKey();
}

// Validate, size the workspace, upload the per-call parameters and enqueue
// (or replay) the run.  Results stay on the device.  tols / ksteps (either may
// be null: tol / maxsteps for every shift) give each shift its own stop
// tolerance and step limit.
int run_async(evc_ctx* ctx, const double* shifts, int S, int m, int maxsteps, double tol,
              uint64_t seed, const double* tols = nullptr, const int* ksteps = nullptr)
{
    if (!ctx) return EVC_EINVAL;
    if (!shifts || S < 1) return fail(ctx, EVC_EINVAL, "need at least one shift");
    if (m < 1) return fail(ctx, EVC_EINVAL, "nprobe must be >= 1 (got %d)", m);
    if (!ksteps && (maxsteps < 1 || maxsteps > EVC_MAX_STEPS))
        return fail(ctx, EVC_EINVAL, "maxsteps must be in [1, %d] (got %d)", EVC_MAX_STEPS, maxsteps);
    if ((int64_t)S * m > (int64_t)1 << 26) return fail(ctx, EVC_EINVAL, "too many columns");
    if ((uint64_t)m + CW > ((uint64_t)1 << 32)) return fail(ctx, EVC_EINVAL, "nprobe too large");
    if (((int64_t)S * m + CW - 1) / CW > 65535)
        return fail(ctx, EVC_EINVAL, "at most 65535*32 (shift, probe) columns per call");
    for (int s = 0; s < S; ++s)
        if (!std::isfinite(shifts[s])) return fail(ctx, EVC_EINVAL, "shift %d is not finite", s);
    if (!std::isfinite(tol)) return fail(ctx, EVC_EINVAL, "tol is not finite");
    int kreq = ksteps ? 0 : maxsteps;
    for (int s = 0; ksteps && s < S; ++s) {
        if (ksteps[s] < 1 || ksteps[s] > EVC_MAX_STEPS)
            return fail(ctx, EVC_EINVAL, "maxsteps of shift %d must be in [1, %d]", s, EVC_MAX_STEPS);
        kreq = std::max(kreq, ksteps[s]);
    }
    for (int s = 0; tols && s < S; ++s)
        if (!std::isfinite(tols[s])) return fail(ctx, EVC_EINVAL, "tol of shift %d is not finite", s);
    const int kmax = (int)std::min<int64_t>(kreq, ctx->n);
    if (ctx->method == EVC_METHOD_ARNOLDI) {
        if (kmax > kArnoldiMaxSteps)
            return fail(ctx, EVC_EINVAL, "the Arnoldi method runs at most %d steps (got %d)",
                        kArnoldiMaxSteps, kmax);
        if (ctx->quad_rule != EVC_QUAD_GAUSS)
            return fail(ctx, EVC_EUNSUPPORTED, "the averaged Gauss rule is a Lanczos quadrature");
        if (ctx->tinv_lanczos)
            return fail(ctx, EVC_EUNSUPPORTED,
                        "the T^-1-inner-product process is a Lanczos method (EVC_OPT_TINV_LANCZOS)");
    }
    if (ctx->tinv_lanczos && ctx->prec == EVC_PREC_CHEB_KINETIC)
        return fail(ctx, EVC_EUNSUPPORTED,
                    "the T^-1-inner-product process needs a diagonal T (Jacobi): its start vector "
                    "z_1 = M^-1 q_1 would need a solve with p_d(K)");
    Layout L = layout(ctx, S, m, kmax);
    if (L.total > ctx->ws_bytes) {
        if (!ctx->ws_owned && ctx->ws)
            return fail(ctx, EVC_ENOMEM, "workspace too small: need %zu bytes, have %zu", L.total,
                        ctx->ws_bytes);
        drop_graph(ctx);
        if (ctx->ws) cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->ws, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, EVC_ENOMEM, "cudaMalloc of %zu bytes failed: %s", L.total,
                        cudaGetErrorString(e));
        }
        ctx->ws_bytes = L.total;
        ctx->ws_owned = true;
    }
    Run r{};
    void* work = nullptr;
    carve(ctx, S, m, kmax, static_cast<char*>(ctx->ws), r, &work);

    // per-call parameters: sigma / shift_of / probe_id per column; shifts, stop
    // tolerance and step limit per shift; operator shifts; seed
    const size_t pbytes = (size_t)L.ncol * (8 + 8 + 4) + (size_t)S * (8 + 8 + 4 + 8) + 64;
    // the previous call's parameter copies must have left the staging buffer
    if (ctx->param_ev) CU(cudaEventSynchronize(ctx->param_ev));
    int rc = ensure_pinned(ctx, &ctx->pinned, &ctx->pinned_bytes, pbytes);
    if (rc) return rc;
    char* h = static_cast<char*>(ctx->pinned);
    double* hsig = reinterpret_cast<double*>(h);
    int64_t* hpid = reinterpret_cast<int64_t*>(h + (size_t)L.ncol * 8);
    int* hsh = reinterpret_cast<int*>(h + (size_t)L.ncol * 16);
    double* hshifts = reinterpret_cast<double*>(h + (size_t)L.ncol * 20);
    double* hstol = hshifts + S;
    double* hops = hstol + S;
    int* hsk = reinterpret_cast<int*>(hops + S);
    uint64_t* hseed = reinterpret_cast<uint64_t*>(h + (((size_t)L.ncol * 20 + (size_t)S * 28 + 7) & ~(size_t)7));
    const int ncr = r.ncol_real;     // Lanczos columns: S*m, or m in shared mode
    for (int c = 0; c < L.ncol; ++c) {
        const bool real = c < ncr;
        // shared mode: every column runs on A itself (operator shift 0)
        const int s = r.shared ? 0 : (real ? c / m : S - 1);
        hsh[c] = s;
        hsig[c] = r.shared ? 0.0 : shifts[s];
        // probe ids probe_offset + j; padding columns run extra probes, ignored
        hpid[c] = ctx->probe_offset + (real ? c % m : (int64_t)m + (c - ncr));
    }
    bool adaptive = false;
    for (int s = 0; s < S; ++s) {
        hshifts[s] = shifts[s];
        hstol[s] = tols ? tols[s] : tol;
        hsk[s] = (int)std::min<int64_t>(ksteps ? ksteps[s] : maxsteps, ctx->n);
        adaptive |= hstol[s] > 0.0 || hsk[s] < kmax;
    }
    for (int s = 0; s < r.Sop; ++s) hops[s] = r.shared ? 0.0 : shifts[s];
    *hseed = seed;
    CU(cudaMemcpyAsync(r.sigma, hsig, (size_t)L.ncol * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.probe_id, hpid, (size_t)L.ncol * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.shift_of, hsh, (size_t)L.ncol * 4, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.shifts, hshifts, (size_t)S * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.stol, hstol, (size_t)S * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.skmax, hsk, (size_t)S * 4, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.opshift, hops, (size_t)r.Sop * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(r.seed, hseed, 8, cudaMemcpyHostToDevice, ctx->stream));
    if (!ctx->param_ev) CU(cudaEventCreateWithFlags(&ctx->param_ev, cudaEventDisableTiming));
    CU(cudaEventRecord(ctx->param_ev, ctx->stream));

    auto enqueue = [&]() -> int {
        ctx->recs.clear();
        ctx->evnext = 0;
        return ctx->tsize == 4 ? enqueue_all<float>(ctx, r, work, adaptive)
                               : enqueue_all<double>(ctx, r, work, adaptive);
    };
    if (ctx->use_graph) {
        GraphKey k;
        k.S = S;
        k.m = m;
        k.kmax = kmax;
        k.adaptive = adaptive;
        k.prec_version = ctx->prec_version;
        k.profile = ctx->profile;
        k.ws = ctx->ws;
        k.ws_bytes = ctx->ws_bytes;
        k.shared = r.shared;
        k.tinv = r.tinv;
        if (!(ctx->gexec && k == ctx->gkey)) {
            drop_graph(ctx);
            cudaGraph_t g = nullptr;
            NvtxRange nv("evc: capture the count's graph");
            CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue();
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess)
                return fail(ctx, EVC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&ctx->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ctx->gexec = nullptr;
                return fail(ctx, EVC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
            }
            ctx->gkey = k;
        }
        NvtxRange nv("evc: launch the count's graph");
        CU(cudaGraphLaunch(ctx->gexec, ctx->stream));
    } else {
        NvtxRange nv("evc: enqueue the count (no graph)");
        rc = enqueue();
        if (rc) return rc;
    }
    ctx->run = r;
    ctx->have_run = true;
    return EVC_OK;
}

int check_device_error(evc_ctx* ctx)
{
    int herr = 0;
    CU(cudaMemcpyAsync(&herr, ctx->run.err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (herr == DERR_NUMERIC)
        return fail(ctx, EVC_ENUMERIC, "non-finite alpha/beta or tridiagonal eigensolver failure");
    if (herr == DERR_TIMEOUT)
        return fail(ctx, EVC_ETIMEOUT, "a bounded device wait gave up (results are invalid)");
    if (herr == DERR_BOUNDS)
        return fail(ctx, EVC_ECUDA, "a bulk copy failed its bounds/alignment check (results are invalid)");
    if (herr) return fail(ctx, EVC_ECUDA, "device error flag %d", herr);
    return EVC_OK;
}

int validate_csr_host(evc_ctx* ctx, const evc_csr* A)
{
    const int64_t n = A->n, nnz = A->nnz;
    if (A->row_ptr[0] != 0 || A->row_ptr[n] != nnz)
        return fail(ctx, EVC_EINVAL, "row_ptr must start at 0 and end at nnz");
    for (int64_t r = 0; r < n; ++r)
        if (A->row_ptr[r + 1] < A->row_ptr[r]) return fail(ctx, EVC_EINVAL, "row_ptr decreases at %lld", (long long)r);
    for (int64_t k = 0; k < nnz; ++k)
        if (A->col[k] < 0 || A->col[k] >= n) return fail(ctx, EVC_EINVAL, "column index out of range at %lld", (long long)k);
    // symmetry: sorted (r, c, v) triplets against sorted (c, r, v)
    struct E { int64_t a, b; double v; };
    std::vector<E> x((size_t)nnz), y((size_t)nnz);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t k = A->row_ptr[r]; k < A->row_ptr[r + 1]; ++k) {
            const double v = A->val_is_fp32 ? (double)static_cast<const float*>(A->val)[k]
                                            : static_cast<const double*>(A->val)[k];
            if (!std::isfinite(v)) return fail(ctx, EVC_EINVAL, "non-finite value at %lld", (long long)k);
            x[k] = E{r, A->col[k], v};
            y[k] = E{A->col[k], r, v};
        }
    auto lt = [](const E& p, const E& q) { return p.a != q.a ? p.a < q.a : p.b < q.b; };
    std::sort(x.begin(), x.end(), lt);
    std::sort(y.begin(), y.end(), lt);
    // sum duplicates then compare
    auto fold = [](std::vector<E>& v) {
        size_t o = 0;
        for (size_t i = 0; i < v.size(); ++i) {
            if (o && v[o - 1].a == v[i].a && v[o - 1].b == v[i].b) v[o - 1].v += v[i].v;
            else v[o++] = v[i];
        }
        v.resize(o);
    };
    fold(x);
    fold(y);
    if (x.size() != y.size()) return fail(ctx, EVC_EINVAL, "matrix is not structurally symmetric");
    for (size_t i = 0; i < x.size(); ++i) {
        if (x[i].a != y[i].a || x[i].b != y[i].b)
            return fail(ctx, EVC_EINVAL, "matrix is not structurally symmetric");
        const double tolv = 1e-12 * std::max(std::fabs(x[i].v), std::fabs(y[i].v));
        if (std::fabs(x[i].v - y[i].v) > tolv) return fail(ctx, EVC_EINVAL, "matrix is not symmetric");
    }
    return EVC_OK;
}

evc_ctx* new_ctx(int precision, void* stream)
{
    evc_ctx* c = new (std::nothrow) evc_ctx();
    if (!c) return nullptr;
    c->precision = precision;
    c->tsize = precision == EVC_MIXED ? 4 : 8;
    c->stream = static_cast<cudaStream_t>(stream);
    if (!c->stream) {
        // The legacy default stream cannot be captured into a graph: run on a
        // private blocking stream, which the legacy stream still orders with.
        if (cudaStreamCreate(&c->stream) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return nullptr;
        }
        c->own_stream = true;
    }
    return c;
}

}  // namespace

// A context that computes on the same matrix and preconditioner as src, on a
// stream of its own (non-blocking), without a workspace; the matrix arrays
// are borrowed from src, which must outlive it.  Used by the request server
// so that several launches on one matrix can be in flight at once.
evc_ctx* evc::clone_context(const evc_ctx* src)
{
    evc_ctx* c = new (std::nothrow) evc_ctx();
    if (!c) return nullptr;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return nullptr;
    }
    c->own_stream = true;
    c->op = src->op;
    c->precision = src->precision;
    c->tsize = src->tsize;
    c->n = src->n;
    c->csr = src->csr;
    c->nnz = src->nnz;
    c->val_fp32 = src->val_fp32;
    c->sten = src->sten;
    c->prec = src->prec;
    c->jac_eps = src->jac_eps;
    c->cheb_degree = src->cheb_degree;
    c->cheb_c = src->cheb_c;
    c->cheb_a = src->cheb_a;
    c->cheb_b = src->cheb_b;
    c->cheb_coef = src->cheb_coef;
    c->cheb_fac = src->cheb_fac;
    c->cheb_g = src->cheb_g;
    c->cheb_sign = src->cheb_sign;
    c->cheb_form = src->cheb_form;
    c->basis_bf16 = src->basis_bf16;
    c->reorth_rows = src->reorth_rows;
    c->sten_groups = src->sten_groups;
    c->method = src->method;
    c->shared_krylov = src->shared_krylov;
    c->tinv_lanczos = src->tinv_lanczos;
    c->quad_rule = src->quad_rule;
    c->min_steps = src->min_steps;
    c->probe_offset = src->probe_offset;
    c->use_graph = false;
    return c;
}

cudaStream_t evc::ctx_stream(const evc_ctx* c) { return c->stream; }
int evc::shares_krylov(const evc_ctx* c, int nshift) { return use_shared(c, nshift) ? 1 : 0; }

// ================================================================== C ABI

extern "C" {

int evc_version(void) { return 10000; }

int evc_cheb_kinetic(int order, double h, int degree, double c, int N, double* info,
                     double* coef, double* factors, int* nfac)
{
    if (!info || !coef || !factors || !nfac || N < 0) return EVC_EINVAL;
    ChebSetup cs;
    if (cheb_setup(order, h, degree, c, N, cs)) return EVC_EINVAL;
    info[0] = cs.a;
    info[1] = cs.b;
    info[2] = N > 0 ? cs.pmin : 0.0;
    info[3] = cs.g;
    info[4] = cs.sign;
    for (int j = 0; j <= degree; ++j) coef[j] = cs.coef[j];
    *nfac = (int)cs.fac.size();
    for (size_t f = 0; f < cs.fac.size(); ++f) {
        factors[3 * f] = cs.fac[f].re;
        factors[3 * f + 1] = cs.fac[f].im;
        factors[3 * f + 2] = cs.fac[f].pair ? 1.0 : 0.0;
    }
    return EVC_OK;
}

int evc_create_csr(const evc_csr* A, int precision, void* stream, evc_ctx** out)
{
    if (!out) return EVC_EINVAL;
    *out = nullptr;
    if (!A || (precision != EVC_FP64 && precision != EVC_MIXED)) return EVC_EINVAL;
    if (A->n < 1 || A->n >= ((int64_t)1 << 31) || A->nnz < 0 || !A->row_ptr ||
        (A->nnz > 0 && (!A->col || !A->val)))
        return EVC_EINVAL;
    evc_ctx* ctx = new_ctx(precision, stream);
    if (!ctx) return EVC_ENOMEM;
    ctx->op = OP_CSR;
    ctx->n = A->n;
    ctx->nnz = A->nnz;
    int rc = EVC_OK;
    if (!A->on_device && A->check) rc = validate_csr_host(ctx, A);
    auto cleanup = [&](int code) {
        evc_destroy(ctx);
        return code;
    };
    if (rc) return cleanup(rc);
    const int64_t n = A->n, nnz = A->nnz;
    auto dmalloc = [&](void** p, size_t b) -> int {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(b, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return EVC_ENOMEM;
        }
        return EVC_OK;
    };
    if (A->on_device) {
        ctx->csr.row_ptr = A->row_ptr;
        ctx->csr.col = A->col;
    } else {
        if (dmalloc(&ctx->own_rowptr, (n + 1) * 8) || dmalloc(&ctx->own_col, nnz * 4))
            return cleanup(EVC_ENOMEM);
        if (cudaMemcpyAsync(ctx->own_rowptr, A->row_ptr, (n + 1) * 8, cudaMemcpyHostToDevice, ctx->stream) ||
            cudaMemcpyAsync(ctx->own_col, A->col, nnz * 4, cudaMemcpyHostToDevice, ctx->stream))
            return cleanup(EVC_ECUDA);
        ctx->csr.row_ptr = static_cast<const int64_t*>(ctx->own_rowptr);
        ctx->csr.col = static_cast<const int32_t*>(ctx->own_col);
    }
    ctx->csr.n = n;
    ctx->csr.nnz = nnz;
    ctx->val_fp32 = A->val_is_fp32 ? 1 : 0;
    if (dmalloc(reinterpret_cast<void**>(&ctx->own_diag), n * 8)) return cleanup(EVC_ENOMEM);
    ctx->csr.diag = ctx->own_diag;
    // the FP64 diagonal comes from the values as given (float64 input stays
    // float64 there even when the context stores float32 values)
    const bool same = (A->val_is_fp32 ? 4u : 8u) == ctx->tsize;
    if (A->on_device && same) {
        ctx->csr.val = A->val;
        csr_diag_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, ctx->stream>>>(
            ctx->csr.row_ptr, ctx->csr.col, A->val, A->val_is_fp32, ctx->own_diag, n);
        if (cudaGetLastError() != cudaSuccess) return cleanup(EVC_ECUDA);
    } else {
        if (dmalloc(&ctx->own_val, nnz * ctx->tsize)) return cleanup(EVC_ENOMEM);
        rc = upload_values(ctx, ctx->own_val, A->val, nnz, A->val_is_fp32, A->on_device,
                           ctx->own_diag);
        if (rc) return cleanup(rc);
        release_stage(ctx);   // kept only by evc_set_values, for repeated updates
        ctx->csr.val = ctx->own_val;
    }
    // visit order of the rows: by decreasing length, so the rows that share a
    // warp in the operator kernel have similar lengths
    {
        std::vector<int64_t> rp((size_t)n + 1);
        if (A->on_device) {
            if (cudaMemcpy(rp.data(), A->row_ptr, (n + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                return cleanup(EVC_ECUDA);
        } else {
            memcpy(rp.data(), A->row_ptr, (n + 1) * 8);
        }
        std::vector<int32_t> perm((size_t)n);
        for (int64_t r = 0; r < n; ++r) perm[r] = (int32_t)r;
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
            return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
        });
        if (dmalloc(reinterpret_cast<void**>(&ctx->own_perm), n * 4)) return cleanup(EVC_ENOMEM);
        if (cudaMemcpyAsync(ctx->own_perm, perm.data(), n * 4, cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess)
            return cleanup(EVC_ECUDA);
        ctx->csr.perm = ctx->own_perm;
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cleanup(EVC_ECUDA);
    }
    *out = ctx;
    return EVC_OK;
}

int evc_create_stencil(int N, double h, int order, const void* V, int V_is_fp32, int on_device,
                       int precision, void* stream, evc_ctx** out)
{
    if (!out) return EVC_EINVAL;
    *out = nullptr;
    if ((precision != EVC_FP64 && precision != EVC_MIXED) || !V || !(h > 0.0) ||
        !std::isfinite(h) || (order != 2 && order != 4))
        return EVC_EINVAL;
    if (N < (order == 2 ? 2 : 5) || (int64_t)N * N * N >= ((int64_t)1 << 31)) return EVC_EINVAL;
    evc_ctx* ctx = new_ctx(precision, stream);
    if (!ctx) return EVC_ENOMEM;
    ctx->op = OP_STENCIL;
    ctx->n = (int64_t)N * N * N;
    StencilOp& s = ctx->sten;
    s.N = N;
    s.order = order;
    s.h = h;
    const double ih2 = 1.0 / (h * h);
    if (order == 2) {
        s.c1 = -0.5 * ih2;
        s.c2 = 0.0;
        s.cd = 3.0 * ih2;
    } else {
        s.c1 = -16.0 / 24.0 * ih2;
        s.c2 = 1.0 / 24.0 * ih2;
        s.cd = 90.0 / 24.0 * ih2;
    }
    const bool same = (V_is_fp32 ? 4u : 8u) == ctx->tsize;
    if (on_device && same) {
        s.V = V;
    } else {
        if (cudaMalloc(&ctx->own_V, ctx->n * ctx->tsize) != cudaSuccess) {
            cudaGetLastError();
            evc_destroy(ctx);
            return EVC_ENOMEM;
        }
        ctx->val_fp32 = V_is_fp32 ? 1 : 0;
        int rc = upload_values(ctx, ctx->own_V, V, ctx->n, V_is_fp32, on_device);
        if (rc == EVC_OK) rc = release_stage(ctx);
        if (rc == EVC_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = EVC_ECUDA;
        if (rc) {
            evc_destroy(ctx);
            return rc;
        }
        s.V = ctx->own_V;
    }
    *out = ctx;
    return EVC_OK;
}

int evc_set_values(evc_ctx* ctx, const void* values, int on_device)
{
    if (!ctx || !values) return EVC_EINVAL;
    void* dst = ctx->op == OP_STENCIL ? ctx->own_V : ctx->own_val;
    if (!dst) return fail(ctx, EVC_EINVAL, "values were borrowed at creation; update them in place");
    const int64_t cnt = ctx->op == OP_STENCIL ? ctx->n : ctx->nnz;
    // the values come in the type given at creation
    return upload_values(ctx, dst, values, cnt, ctx->val_fp32, on_device,
                         ctx->op == OP_CSR ? ctx->own_diag : nullptr);
}

int evc_set_precond(evc_ctx* ctx, int kind, double param0, double param1)
{
    if (!ctx) return EVC_EINVAL;
    NvtxRange nv("evc: set the preconditioner");
    if (kind == EVC_PREC_IDENTITY) {
        ctx->prec = kind;
    } else if (kind == EVC_PREC_JACOBI) {
        if (!(param0 > 0.0) || !std::isfinite(param0))
            return fail(ctx, EVC_EINVAL, "Jacobi eps must be > 0");
        ctx->prec = kind;
        ctx->jac_eps = param0;
    } else if (kind == EVC_PREC_CHEB_KINETIC) {
        if (ctx->op != OP_STENCIL)
            return fail(ctx, EVC_EUNSUPPORTED, "the kinetic Chebyshev preconditioner needs a stencil context");
        const int d = (int)param0;
        if ((double)d != param0)
            return fail(ctx, EVC_EINVAL, "Chebyshev degree must be an integer in [1, 32]");
        const StencilOp& s = ctx->sten;
        ChebSetup cs;
        if (const char* why = cheb_setup(s.order, s.h, d, param1, s.N, cs))
            return fail(ctx, EVC_EINVAL, "%s", why);
        if (!(cs.pmin > 0.0))
            return fail(ctx, EVC_EINVAL, "Chebyshev preconditioner not positive on spec(K) (min %g)", cs.pmin);
        ctx->prec = kind;
        ctx->cheb_degree = d;
        ctx->cheb_c = param1;
        ctx->cheb_a = cs.a;
        ctx->cheb_b = cs.b;
        ctx->cheb_coef = cs.coef;
        ctx->cheb_fac = cs.fac;          // empty: Clenshaw's recurrence only
        ctx->cheb_g = cs.g;
        ctx->cheb_sign = cs.sign;
    } else {
        return fail(ctx, EVC_EINVAL, "unknown preconditioner kind %d", kind);
    }
    ++ctx->prec_version;
    return EVC_OK;
}

size_t evc_workspace_bytes(const evc_ctx* ctx, int nshift, int nprobe, int maxsteps)
{
    if (!ctx || nshift < 1 || nprobe < 1 || maxsteps < 1 || maxsteps > EVC_MAX_STEPS) return 0;
    const int kmax = (int)std::min<int64_t>(maxsteps, ctx->n);
    return layout(ctx, nshift, nprobe, kmax).total;
}

int evc_set_workspace(evc_ctx* ctx, void* dptr, size_t bytes)
{
    if (!ctx) return EVC_EINVAL;
    if (dptr && ((uintptr_t)dptr & 255)) return fail(ctx, EVC_EINVAL, "workspace must be 256-byte aligned");
    drop_graph(ctx);
    if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
    ctx->ws = dptr;
    ctx->ws_bytes = dptr ? bytes : 0;
    ctx->ws_owned = false;
    ctx->have_run = false;
    return EVC_OK;
}

int evc_count_slices_async(evc_ctx* ctx, const double* shifts, int nshift, int nprobe,
                           int maxsteps, double tol, uint64_t seed, double* d_n_below,
                           double* d_quad, int* d_steps)
{
    int rc = run_async(ctx, shifts, nshift, nprobe, maxsteps, tol, seed);
    if (rc) return rc;
    const Run& r = ctx->run;
    if (d_quad)
        CU(cudaMemcpyAsync(d_quad, r.quad_final, (size_t)r.nq * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_n_below)
        CU(cudaMemcpyAsync(d_n_below, r.Lfinal, (size_t)r.S * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_steps)
        CU(cudaMemcpyAsync(d_steps, r.steps, (size_t)r.S * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return EVC_OK;
}

int evc_sync(evc_ctx* ctx)
{
    if (!ctx) return EVC_EINVAL;
    if (!ctx->have_run) {
        CU(cudaStreamSynchronize(ctx->stream));
        return EVC_OK;
    }
    return check_device_error(ctx);
}

}  // extern "C"

namespace {
// Copy the last run's results to the caller's host buffers (any may be null)
// after checking the device's error flag.
int fetch_results(evc_ctx* ctx, double* n_below, double* per_probe_quad, int* steps_used)
{
    int rc;
    const Run& r = ctx->run;
    const size_t need = (size_t)r.nq * 8 + (size_t)r.S * 12 + 64;
    rc = ensure_pinned(ctx, &ctx->pinres, &ctx->pinres_bytes, need);
    if (rc) return rc;
    char* h = static_cast<char*>(ctx->pinres);
    double* hq = reinterpret_cast<double*>(h);
    double* hL = hq + r.nq;
    int* hs = reinterpret_cast<int*>(hL + r.S);
    CU(cudaMemcpyAsync(hq, r.quad_final, (size_t)r.nq * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(hL, r.Lfinal, (size_t)r.S * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(hs, r.steps, (size_t)r.S * 4, cudaMemcpyDeviceToHost, ctx->stream));
    rc = check_device_error(ctx);
    if (rc) return rc;
    if (per_probe_quad) memcpy(per_probe_quad, hq, (size_t)r.nq * 8);
    if (n_below) memcpy(n_below, hL, (size_t)r.S * 8);
    if (steps_used) memcpy(steps_used, hs, (size_t)r.S * 4);
    return EVC_OK;
}
}  // namespace

int evc::count_slices_each(evc_ctx* ctx, const double* shifts, int nshift, int nprobe,
                           const int* maxsteps, const double* tol, uint64_t seed, double* n_below,
                           double* per_probe_quad, int* steps_used)
{
    if (!maxsteps || !tol) return fail(ctx, EVC_EINVAL, "per-shift step limits and tolerances");
    int rc = run_async(ctx, shifts, nshift, nprobe, 0, 0.0, seed, tol, maxsteps);
    if (rc) return rc;
    return fetch_results(ctx, n_below, per_probe_quad, steps_used);
}

extern "C" {

int evc_count_slices(evc_ctx* ctx, const double* shifts, int nshift, int nprobe, int maxsteps,
                     double tol, uint64_t seed, double* n_below, double* per_probe_quad,
                     int* steps_used)
{
    int rc = run_async(ctx, shifts, nshift, nprobe, maxsteps, tol, seed);
    if (rc) return rc;
    return fetch_results(ctx, n_below, per_probe_quad, steps_used);
}


int evc_count(evc_ctx* ctx, double xi, double eta, int nprobe, int maxsteps, double tol,
              uint64_t seed, double* estimate, double* per_probe_quad, int* steps_used)
{
    if (!ctx) return EVC_EINVAL;
    if (!(xi < eta)) return fail(ctx, EVC_EINVAL, "need xi < eta");
    const double sh[2] = {xi, eta};
    double L[2];
    int rc = evc_count_slices(ctx, sh, 2, nprobe, maxsteps, tol, seed, L, per_probe_quad, steps_used);
    if (rc) return rc;
    if (estimate) *estimate = L[1] - L[0];
    return EVC_OK;
}

int evc_get_tridiag(evc_ctx* ctx, double* alpha, double* beta, int* kdone)
{
    if (ctx && ctx->have_run && ctx->run.arnoldi)
        return fail(ctx, EVC_EUNSUPPORTED, "the last call ran the Arnoldi method: no tridiagonal");
    if (!ctx) return EVC_EINVAL;
    if (!ctx->have_run) return fail(ctx, EVC_EINVAL, "no previous run");
    const Run& r = ctx->run;
    const int K = r.kmax, nc = r.ncol;
    std::vector<double> a((size_t)K * nc), b((size_t)(K + 1) * nc), sh(r.S);
    std::vector<int> kd(nc), st(r.S);
    CU(cudaMemcpyAsync(a.data(), r.alpha, a.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(b.data(), r.beta, b.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(kd.data(), r.kdone, kd.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(sh.data(), r.shifts, sh.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(st.data(), r.steps, st.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    // output column c = s*m + j; in shared mode it is the run's column j, with
    // J(A - tau_s I) = J(A) - tau_s I, up to the step the shift stopped at
    for (int c = 0; c < r.nq; ++c) {
        const int s = c / r.m, lc = r.shared ? c % r.m : c;
        const int done = r.shared ? (kd[lc] ? std::min(kd[lc], st[s]) : st[s]) : kd[lc];
        const double off = r.shared ? sh[s] : 0.0;
        if (kdone) kdone[c] = done;
        for (int i = 0; i < K; ++i) {
            if (alpha) alpha[(size_t)c * K + i] = i < done ? a[(size_t)i * nc + lc] - off : 0.0;
            if (beta) beta[(size_t)c * (K + 1) + i] = i <= done ? b[(size_t)i * nc + lc] : 0.0;
        }
        if (beta) beta[(size_t)c * (K + 1) + K] = K <= done ? b[(size_t)K * nc + lc] : 0.0;
    }
    return EVC_OK;
}

int evc_get_quad_bound(evc_ctx* ctx, double* log10_bound)
{
    if (!ctx) return EVC_EINVAL;
    if (!log10_bound) return fail(ctx, EVC_EINVAL, "null output");
    if (!ctx->have_run) return fail(ctx, EVC_EINVAL, "no previous run");
    const int K = ctx->run.kmax, nq = ctx->run.nq;
    const double vn2 = (double)ctx->run.n;     // ||v||^2 of a Rademacher probe
    std::vector<double> b((size_t)(K + 1) * nq);
    std::vector<int> kd(nq);
    const int rc = evc_get_tridiag(ctx, nullptr, b.data(), kd.data());
    if (rc) return rc;
    for (int c = 0; c < nq; ++c) {
        const int k = kd[c];
        if (k < 1) {
            log10_bound[c] = std::nan("");
            continue;
        }
        // log10 of ||v||^2 prod_{j=2}^{k+1} beta_j^2 / (2k)!
        double s = std::log10(vn2) - std::lgamma(2.0 * k + 1.0) / std::log(10.0);
        bool exact = false;
        for (int j = 2; j <= k + 1; ++j) {
            const double bj = b[(size_t)c * (K + 1) + (j - 1)];
            if (!(bj > 0.0)) {
                exact = true;
                break;
            }
            s += 2.0 * std::log10(bj);
        }
        log10_bound[c] = exact ? -INFINITY : s;
    }
    return EVC_OK;
}

int evc_set_option(evc_ctx* ctx, int option, int64_t value)
{
    if (!ctx) return EVC_EINVAL;
    if (option == EVC_OPT_GRAPH) {
        ctx->use_graph = value != 0;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_PROFILE) {
        ctx->profile = value != 0;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_MIN_STEPS) {
        if (value < 1 || value > EVC_MAX_STEPS)
            return fail(ctx, EVC_EINVAL, "min steps must be in [1, %d]", EVC_MAX_STEPS);
        ctx->min_steps = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_PROBE_OFFSET) {
        if (value < 0 || value > ((int64_t)1 << 31))
            return fail(ctx, EVC_EINVAL, "probe offset must be in [0, 2^31]");
        ctx->probe_offset = value;     // a per-call upload, no graph change
        return EVC_OK;
    }
    if (option == EVC_OPT_METHOD) {
        if (value != EVC_METHOD_LANCZOS && value != EVC_METHOD_ARNOLDI)
            return fail(ctx, EVC_EINVAL, "unknown method %lld", (long long)value);
        ctx->method = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_REORTH_ROWS) {
        if (value != 0 && (value < kMinReorthRows || value > ((int64_t)1 << 30)))
            return fail(ctx, EVC_EINVAL, "reorthogonalisation rows per block must be >= %d", kMinReorthRows);
        if (choose_nblk(ctx->n, (int)value) > reorth_max_blocks(ctx->n))
            return fail(ctx, EVC_EINVAL, "at most %d reorthogonalisation blocks per chunk for n = %lld",
                        reorth_max_blocks(ctx->n), (long long)ctx->n);
        ctx->reorth_rows = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_STENCIL_ZB) {
        if (ctx->op != OP_STENCIL) return fail(ctx, EVC_EINVAL, "not a stencil context");
        if (value < 0 || value > 65536) return fail(ctx, EVC_EINVAL, "z planes per block must be in [0, 65536]");
        ctx->sten.zb = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_STENCIL_PATCH) {
        if (ctx->op != OP_STENCIL) return fail(ctx, EVC_EINVAL, "not a stencil context");
        if (value != 1 && value != 2 && value != 3)
            return fail(ctx, EVC_EINVAL, "stencil patch must be 1, 2 or 3");
        ctx->sten.patch = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_STENCIL_GROUPS) {
        if (ctx->op != OP_STENCIL) return fail(ctx, EVC_EINVAL, "not a stencil context");
        if (value < 1 || value > kMaxStencilGroups)
            return fail(ctx, EVC_EINVAL, "stencil chunk groups must be in [1, %d]", kMaxStencilGroups);
        ctx->sten_groups = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_SHARED_KRYLOV) {
        if (value != 0 && value != 1) return fail(ctx, EVC_EINVAL, "shared Krylov option must be 0 or 1");
        ctx->shared_krylov = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_TINV_LANCZOS) {
        if (value != 0 && value != 1) return fail(ctx, EVC_EINVAL, "T^-1 Lanczos option must be 0 or 1");
        ctx->tinv_lanczos = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_CSR_THREADS) {
        if (ctx->op != OP_CSR) return fail(ctx, EVC_EINVAL, "not a CSR context");
        if (value != 128 && value != 256 && value != 512)
            return fail(ctx, EVC_EINVAL, "CSR threads per block must be 128, 256 or 512");
        ctx->csr.threads = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_BASIS_BF16) {
        if (value != 0 && value != 1) return fail(ctx, EVC_EINVAL, "BF16 basis option must be 0 or 1");
        if (value && ctx->precision != EVC_MIXED)
            return fail(ctx, EVC_EINVAL, "BF16 basis storage applies to EVC_MIXED contexts only");
        ctx->basis_bf16 = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_CHEB_FORM) {
        if (value != EVC_CHEB_FACTORED && value != EVC_CHEB_CLENSHAW)
            return fail(ctx, EVC_EINVAL, "unknown Chebyshev evaluation form %lld", (long long)value);
        ctx->cheb_form = (int)value;
        ++ctx->prec_version;
        drop_graph(ctx);
        return EVC_OK;
    }
    if (option == EVC_OPT_QUADRATURE) {
        if (value != EVC_QUAD_GAUSS && value != EVC_QUAD_GA)
            return fail(ctx, EVC_EINVAL, "unknown quadrature rule %lld", (long long)value);
        ctx->quad_rule = (int)value;
        ++ctx->prec_version;   // part of the captured graph
        drop_graph(ctx);
        return EVC_OK;
    }
    return fail(ctx, EVC_EINVAL, "unknown option %d", option);
}

int evc_get_profile(evc_ctx* ctx, evc_prof_rec* recs, int cap, int* nrec)
{
    if (!ctx) return EVC_EINVAL;
    if (nrec) *nrec = (int)ctx->recs.size();
    if (!recs || cap <= 0) return EVC_OK;
    CU(cudaStreamSynchronize(ctx->stream));
    std::vector<int> nact;
    if (ctx->have_run) {
        nact.resize(ctx->run.kmax + 1);
        CU(cudaMemcpy(nact.data(), ctx->run.nactive, nact.size() * sizeof(int),
                      cudaMemcpyDeviceToHost));
    }
    const int cnt = std::min<int>(cap, (int)ctx->recs.size());
    for (int i = 0; i < cnt; ++i) {
        const evc_ctx::Rec& r = ctx->recs[i];
        recs[i].kind = r.kind;
        recs[i].step = r.step;
        const int act = (ctx->have_run && r.step >= 1 && r.step <= (int)nact.size())
                            ? nact[r.step - 1]
                            : (ctx->have_run ? ctx->run.nchunk : 0);
        recs[i].bytes = r.fixed + r.per_chunk * act;
        float ms = -1.0f;
        if (r.e0 && r.e1) CU(cudaEventElapsedTime(&ms, r.e0, r.e1));
        recs[i].ms = ms;
        recs[i].span = r.span;
        recs[i].reserved = 0;
    }
    return EVC_OK;
}

int evc_autotune(evc_ctx* ctx, int nshift, int nprobe, int maxsteps, evc_tuning* out)
{
    if (!ctx || nshift < 1 || nprobe < 1 || maxsteps < 1) return EVC_EINVAL;
    NvtxRange nv("evc: autotune");
    // short counts of the caller's shape (placeholder shifts: the timing of
    // a fixed number of steps does not depend on them)
    const int kt = std::min(maxsteps, 6);
    const std::vector<double> shifts(nshift, 0.0);
    const bool prof0 = ctx->profile;
    const int rows0 = ctx->reorth_rows, zb0 = ctx->sten.zb, nt0 = ctx->csr.threads,
              pa0 = ctx->sten.patch, gr0 = ctx->sten_groups;
    auto restore = [&](int rc) {
        ctx->profile = prof0;
        ++ctx->prec_version;
        drop_graph(ctx);
        if (rc) {
            ctx->reorth_rows = rows0;
            ctx->sten.zb = zb0;
            ctx->sten.patch = pa0;
            ctx->sten_groups = gr0;
            ctx->csr.threads = nt0;
        }
        return rc;
    };
    ctx->profile = true;
    // device time of the kernel classes in mask (all classes when 0), best of two counts
    auto measure = [&](unsigned mask, double& ms) -> int {
        ms = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            ++ctx->prec_version;     // a fresh graph per configuration
            int rc = evc_count_slices(ctx, shifts.data(), nshift, nprobe, kt, 0.0, 1, nullptr,
                                      nullptr, nullptr);
            if (rc) return rc;
            int nr = 0;
            evc_get_profile(ctx, nullptr, 0, &nr);
            std::vector<evc_prof_rec> recs(nr);
            rc = evc_get_profile(ctx, recs.data(), nr, &nr);
            if (rc) return rc;
            double t = 0.0;
            for (const auto& q : recs)
                if (q.ms > 0 && (mask == 0 || (mask >> q.kind) & 1u)) t += q.ms;
            ms = std::min(ms, t);
        }
        return EVC_OK;
    };
    evc_tuning res{};
    int rc = measure(0, res.ms_before);
    if (rc) return restore(rc);
    // operator pass: z planes per block (stencil) or threads per block (CSR)
    if (ctx->op == OP_STENCIL) {
        const int N = ctx->sten.N;
        std::vector<int> cand;
        for (int zb : {16, 32, 64}) cand.push_back(std::min(zb, N));
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        // points per thread and z planes per block at the current chunk groups
        auto tune_shape = [&]() -> int {
            double best = 1e300;
            int bz = cand[0], bp = 1;
            for (int pa : {1, 2, 3}) {
                if (pa == 2 && N % 2) continue;
                if (pa == 3 && !(ctx->precision == EVC_MIXED ? stencil_tma_eligible<float>(N)
                                                             : stencil_tma_eligible<double>(N)))
                    continue;
                for (int zb : cand) {
                    ctx->sten.zb = zb;
                    ctx->sten.patch = pa;
                    double t;
                    const int e = measure(1u << EVC_K_STENCIL, t);
                    if (e) return e;
                    if (t < best) {
                        best = t;
                        bz = zb;
                        bp = pa;
                    }
                }
            }
            ctx->sten.zb = bz;
            ctx->sten.patch = bp;
            return EVC_OK;
        };
        if ((rc = tune_shape())) return restore(rc);
        // concurrent chunk groups of the operator segment (at most one per chunk)
        const int nchunk = (int)(((int64_t)nshift * nprobe + CW - 1) / CW);
        const int g0 = ctx->sten_groups;
        double best = 1e300;
        int bg = 1;
        for (int g : {1, 2, 4}) {
            if (g > 1 && g > nchunk) continue;
            ctx->sten_groups = g;
            double t;
            if ((rc = measure(1u << EVC_K_STENCIL, t))) return restore(rc);
            if (t < best) {
                best = t;
                bg = g;
            }
        }
        ctx->sten_groups = bg;
        // the launch shape of a pass changes with the groups: shapes again
        if (bg != g0 && (rc = tune_shape())) return restore(rc);
    } else {
        double best = 1e300;
        int bt = 256;
        for (int nt : {128, 256, 512}) {
            ctx->csr.threads = nt;
            double t;
            if ((rc = measure(1u << EVC_K_CSR, t))) return restore(rc);
            if (t < best) {
                best = t;
                bt = nt;
            }
        }
        ctx->csr.threads = bt;
    }
    // reorthogonalisation: rows per block
    {
        double best = 1e300;
        int br = 0;
        int last_nblk = -1;
        for (int rows : {64, 128, 256, 512, 1024, 1728, 3456, 6912, 13824}) {
            const int nb = choose_nblk(ctx->n, rows);
            if (nb == last_nblk || nb > reorth_max_blocks(ctx->n)) continue;
            last_nblk = nb;
            ctx->reorth_rows = rows;
            double t;
            if ((rc = measure((1u << EVC_K_DOTS) | (1u << EVC_K_REDUCE) | (1u << EVC_K_UPDATE), t)))
                return restore(rc);
            if (t < best) {
                best = t;
                br = rows;
            }
        }
        ctx->reorth_rows = br;
    }
    rc = measure(0, res.ms_after);
    if (rc) return restore(rc);
    res.stencil_zb = ctx->op == OP_STENCIL ? ctx->sten.zb : 0;
    res.stencil_patch = ctx->op == OP_STENCIL ? std::max(1, ctx->sten.patch) : 0;
    res.stencil_groups = ctx->op == OP_STENCIL ? ctx->sten_groups : 0;
    res.csr_threads = ctx->op == OP_CSR ? ctx->csr.threads : 0;
    res.reorth_rows = ctx->reorth_rows > 0 ? ctx->reorth_rows : default_reorth_rows(ctx->n);
    res.steps = kt;
    if (out) *out = res;
    return restore(EVC_OK);
}

const char* evc_last_error(const evc_ctx* ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

void evc_destroy(evc_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
    if (ctx->own_rowptr) cudaFree(ctx->own_rowptr);
    if (ctx->own_col) cudaFree(ctx->own_col);
    if (ctx->own_val) cudaFree(ctx->own_val);
    if (ctx->own_diag) cudaFree(ctx->own_diag);
    if (ctx->own_perm) cudaFree(ctx->own_perm);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->own_V) cudaFree(ctx->own_V);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->pinres) cudaFreeHost(ctx->pinres);
    if (ctx->param_ev) cudaEventDestroy(ctx->param_ev);
    for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
    for (cudaStream_t s : ctx->aux)
        if (s) cudaStreamDestroy(s);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
