// C ABI of libdpre: contexts, gauge fields, operator application, the
// device-resident dslash entry point, the launch tuner and kernel timing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace dp {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

#define CUDA_OK(expr)                                                            \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return DP_ERR_CUDA;                                                  \
        }                                                                        \
    } while (0)

void *Ctx::alloc(size_t n)
{
    if (n == 0) n = 256;
    void *p = nullptr;
    if (has_hooks) {
        p = hooks.alloc(n, (void *)stream, hooks.user);
    } else if (cudaMallocFromPoolAsync(&p, n, pool, stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        std::lock_guard<std::mutex> lk(mu);
        allocs[p] = n;
        bytes += n;
    }
    return p;
}

void Ctx::release(void *p)
{
    if (!p) return;
    size_t n = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = allocs.find(p);
        if (it == allocs.end()) return;
        n = it->second;
        bytes -= n;
        allocs.erase(it);
    }
    if (has_hooks)
        hooks.free(p, n, (void *)stream, hooks.user);
    else
        cudaFreeAsync(p, stream);
}

cudaEvent_t Ctx::get_event()
{
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void Ctx::time_begin(const char *name, cudaEvent_t *a, cudaStream_t st)
{
    (void)name;
    *a = nullptr;
    if (!timing || (st && st != stream)) return;
    *a = get_event();
    cudaEventRecord(*a, stream);
}

void Ctx::time_end(const char *name, cudaEvent_t a, cudaStream_t st)
{
    if (!timing || !a || (st && st != stream)) return;
    cudaEvent_t b = get_event();
    cudaEventRecord(b, stream);
    pending.push_back({name, a, b});
    if (pending.size() > 4096) collect_timing();
}

void Ctx::collect_timing()
{
    if (pending.empty()) return;
    cudaStreamSynchronize(stream);
    for (auto &p : pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        Stat &s = stats[p.name];
        s.launches++;
        s.ms += ms;
        event_pool.push_back(p.a);
        event_pool.push_back(p.b);
    }
    pending.clear();
}

Shape Ctx::launch_shape(long long Vh, int prec, int link_fmt, int nrhs)
{
    std::lock_guard<std::mutex> lk(mu);
    auto it = tuned.find(TuneKey{Vh, prec, link_fmt, nrhs});
    if (it != tuned.end()) return it->second;
    Shape sh;
    sh.block = 64;
    sh.rpt = prec == 0 ? 1 : 2;  // FP32: one RHS pair per thread
    sh.stages = 0;
    return sh;
}

std::shared_ptr<Field> find_field(Ctx *c, dp_field f)
{
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->fields.find(f);
    if (it == c->fields.end()) return nullptr;
    return it->second;
}

int inner_link_format(int prec, int compress12)
{
    switch (prec) {
    case DP_PREC_FP64: return LINK_F64_18;
    case DP_PREC_MIXED_FP16: return LINK_H16_12;
    case DP_PREC_MIXED_BF16: return LINK_B16_12;
    default: return compress12 ? LINK_F32_12 : LINK_F32_18;
    }
}

dp_status field_links(Ctx *c, Field &f, int link_fmt, int parity, const void **out)
{
    switch (link_fmt) {
    case LINK_F64_18: *out = f.l64[parity]; return DP_OK;
    case LINK_F32_18: *out = f.l32f[parity]; return DP_OK;
    case LINK_F32_12: *out = f.l32c[parity]; return DP_OK;
    case LINK_H16_12:
    case LINK_B16_12: break;
    case LINK_DF_18: {
        std::lock_guard<std::mutex> lk(f.inv_mu);
        if (!f.ldf[0]) {
            const long long cnt = f.g.Vh * 36;
            float4 *d0 = (float4 *)c->alloc(cnt * sizeof(float4)), *d1 = (float4 *)c->alloc(cnt * sizeof(float4));
            cudaError_t e = (d0 && d1) ? launch_to_df(f.l64[0], d0, cnt, nullptr, 1, 0, c->stream)
                                       : cudaErrorMemoryAllocation;
            if (e == cudaSuccess) e = launch_to_df(f.l64[1], d1, cnt, nullptr, 1, 0, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                c->release(d0);
                c->release(d1);
                set_error("double-float links: %s", cudaGetErrorString(e));
                return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : DP_ERR_CUDA;
            }
            c->launches += 2;
            f.ldf[0] = d0;
            f.ldf[1] = d1;
        }
        *out = f.ldf[parity];
        return DP_OK;
    }
    default: set_error("unknown link format %d", link_fmt); return DP_ERR_INVALID_ARG;
    }
    const int k = link_fmt == LINK_H16_12 ? 0 : 1;
    std::lock_guard<std::mutex> lk(f.inv_mu);
    if (!f.l16[k][0]) {
        void *p0 = c->alloc(links16_bytes(f.g.Vh)), *p1 = c->alloc(links16_bytes(f.g.Vh));
        if (!p0 || !p1) {
            c->release(p0);
            c->release(p1);
            set_error("out of device memory (16-bit links)");
            return DP_ERR_OOM;
        }
        cudaError_t e = launch_pack_links16(f.l64[0], f.g.Vh, link_fmt, p0, c->stream);
        if (e == cudaSuccess) e = launch_pack_links16(f.l64[1], f.g.Vh, link_fmt, p1, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            c->release(p0);
            c->release(p1);
            set_error("packing 16-bit links: %s", cudaGetErrorString(e));
            return DP_ERR_CUDA;
        }
        c->launches += 2;
        f.l16[k][0] = p0;
        f.l16[k][1] = p1;
    }
    *out = f.l16[k][parity];
    return DP_OK;
}

dp_status profile_tables(const dp_profile &p, const Geom &g, int bc_t, const int src[4],
                         double *alpha, double *hop)
{
    const int L[4] = {g.T, g.Lx, g.Ly, g.Lz};
    const int Lm = g.Lmax;
    if (!std::isfinite(p.alpha0)) {
        set_error("profile alpha0 is not finite");
        return DP_ERR_INVALID_ARG;
    }
    for (int mu = 0; mu < 4; mu++) {
        for (int x = 0; x < Lm; x++) alpha[mu * Lm + x] = 1.0;
        for (int x = 0; x < L[mu]; x++) {
            const int rel = ((x - src[mu]) % L[mu] + L[mu]) % L[mu];
            const double h = 0.5 * L[mu];
            double a = 1.0;
            switch (p.kind) {
            case DP_PROF_NONE: a = 1.0; break;
            case DP_PROF_EXP_T: a = mu == 0 ? std::exp(p.alpha0 * rel) : 1.0; break;
            case DP_PROF_COSH_T: a = mu == 0 ? 1.0 / std::cosh(p.alpha0 * (rel - h)) : 1.0; break;
            case DP_PROF_COSH_4D: a = std::cosh(p.alpha0 * (rel - h)); break;
            case DP_PROF_TABLE:
                if (!p.table[mu]) {
                    set_error("TABLE profile without table for direction %d", mu);
                    return DP_ERR_INVALID_ARG;
                }
                a = p.table[mu][x];
                break;
            default: set_error("unknown profile kind %d", p.kind); return DP_ERR_INVALID_ARG;
            }
            if (!(a > 0) || !std::isfinite(a)) {
                set_error("profile value not positive and finite (dir %d, x %d)", mu, x);
                return DP_ERR_INVALID_ARG;
            }
            alpha[mu * Lm + x] = a;
        }
    }
    for (int mu = 0; mu < 4; mu++) {
        for (int x = 0; x < 2 * Lm; x++) hop[mu * 2 * Lm + x] = 0.0;
        for (int x = 0; x < L[mu]; x++) {
            const int xp = (x + 1) % L[mu], xm = (x + L[mu] - 1) % L[mu];
            const double sf = (mu == 0 && x == L[mu] - 1) ? bc_t : 1.0;
            const double sb = (mu == 0 && x == 0) ? bc_t : 1.0;
            const double *a = alpha + mu * Lm;
            hop[(mu * 2 + 0) * Lm + x] = -0.5 * sf * a[x] / a[xp];
            hop[(mu * 2 + 1) * Lm + x] = -0.5 * sb * a[x] / a[xm];
        }
    }
    return DP_OK;
}

CloverInv::~CloverInv()
{
    if (!owner) return;
    for (int p = 0; p < 2; p++) {
        owner->release(inv64[p]);
        owner->release(inv32[p]);
        owner->release(invdf[p]);
    }
}

dp_status clover_inv_df(Ctx *c, Field &f, CloverInv &ci)
{
    std::lock_guard<std::mutex> lk(f.inv_mu);
    if (ci.invdf[0]) return DP_OK;
    const long long Vh = f.g.Vh;
    float4 *d[2] = {(float4 *)c->alloc(Vh * 36 * sizeof(float4)), (float4 *)c->alloc(Vh * 36 * sizeof(float4))};
    if (!d[0] || !d[1]) {
        c->release(d[0]);
        c->release(d[1]);
        set_error("out of device memory (double-float clover inverse)");
        return DP_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < 2 && e == cudaSuccess; p++)
        e = launch_to_df(ci.inv64[p], d[p], Vh * 36, nullptr, 1, 0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->release(d[0]);
        c->release(d[1]);
        set_error("double-float clover inverse: %s", cudaGetErrorString(e));
        return DP_ERR_CUDA;
    }
    c->launches += 2;
    ci.invdf[0] = d[0];
    ci.invdf[1] = d[1];
    return DP_OK;
}

dp_status get_clover_inv(Ctx *c, Field &f, double M, std::shared_ptr<CloverInv> *out)
{
    if (!f.has_clover) {
        set_error("clover term not built: call dp_field_set_csw first");
        return DP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(f.inv_mu);
    for (size_t k = 0; k < f.invs.size(); k++)
        if (f.invs[k]->M == M) {
            auto ci = f.invs[k];  // move to the most-recently-used end
            f.invs.erase(f.invs.begin() + k);
            f.invs.push_back(ci);
            *out = ci;
            return DP_OK;
        }
    auto ci = std::make_shared<CloverInv>();
    ci->owner = c;
    ci->M = M;
    const long long Vh = f.g.Vh;
    for (int p = 0; p < 2; p++) {
        ci->inv64[p] = (double2 *)c->alloc(Vh * 36 * sizeof(double2));
        ci->inv32[p] = (float4 *)c->alloc(Vh * 18 * sizeof(float4));
        if (!ci->inv64[p] || !ci->inv32[p]) {
            set_error("out of device memory (clover inverse)");
            return DP_ERR_OOM;
        }
    }
    int *flag = (int *)c->alloc(sizeof(int));
    if (!flag) {
        set_error("out of device memory (clover inverse)");
        return DP_ERR_OOM;
    }
    int h = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    for (int p = 0; p < 2 && e == cudaSuccess; p++)
        e = launch_clover_invert(f.clov[p], Vh, M, ci->inv64[p], ci->inv32[p], flag, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->release(flag);
    c->launches += 2;
    if (e != cudaSuccess) {
        set_error("clover inverse: %s", cudaGetErrorString(e));
        return DP_ERR_CUDA;
    }
    if (h) {
        set_error("clover block (4+M)+clover is singular or non-finite at M=%g", M);
        return DP_ERR_NONFINITE;
    }
    // the cache keeps the 16 most recently used masses per field
    if (f.invs.size() >= 16) f.invs.erase(f.invs.begin());
    f.invs.push_back(ci);
    *out = ci;
    return DP_OK;
}

dp_status check_opts(const dp_solve_opts *in, dp_solve_opts *out)
{
    dp_solve_opts o{};
    if (in) o = *in;
    if (o.max_iter <= 0) o.max_iter = 20000;
    if (o.prec < DP_PREC_FP64 || o.prec > DP_PREC_MIXED_BF16) {
        set_error("invalid precision %d", o.prec);
        return DP_ERR_INVALID_ARG;
    }
    if (o.solver != DP_SOLVER_BICGSTAB && o.solver != DP_SOLVER_CGNE && o.solver != DP_SOLVER_SAP_GCR) {
        set_error("unknown solver %d", o.solver);
        return DP_ERR_INVALID_ARG;
    }
    if (o.solver == DP_SOLVER_SAP_GCR && o.prec == DP_PREC_FP64) {
        set_error("SAP+GCR runs as the FP32 inner solver: choose a mixed precision");
        return DP_ERR_INVALID_ARG;
    }
    if (o.sap_ncy < 0 || o.sap_ncy > 64 || o.sap_nmr < 0 || o.sap_nmr > 64 || o.gcr_nkv < 0 ||
        o.gcr_nkv > 32) {
        set_error("sap_ncy, sap_nmr in [0, 64], gcr_nkv in [0, 32]");
        return DP_ERR_INVALID_ARG;
    }
    if (o.sap_ncy == 0) o.sap_ncy = 4;
    if (o.sap_nmr == 0) o.sap_nmr = 4;
    if (o.gcr_nkv == 0) o.gcr_nkv = 8;
    if (!(o.inner_tol >= 0) || o.inner_tol >= 1) {
        set_error("inner_tol must be in [0, 1)");
        return DP_ERR_INVALID_ARG;
    }
    // FP32 BiCGStab reliably reduces the residual by 1e-6 before rounding
    // stalls it; two FP64 rounds then reach r = 1e-11
    if (o.inner_tol == 0) o.inner_tol = o.prec == DP_PREC_FP64 ? 0.0 : 1e-6;
    if (o.check_every < 0) o.check_every = 0;
    if (o.outer_df != 0 && o.outer_df != 1) {
        set_error("outer_df must be 0 or 1");
        return DP_ERR_INVALID_ARG;
    }
    if (o.prec == DP_PREC_FP64) o.outer_df = 0;  // the FP64 solver has no separate outer operator
    if (!std::isfinite(o.slice_tol)) {
        set_error("slice_tol must be finite");
        return DP_ERR_INVALID_ARG;
    }
    *out = o;
    return DP_OK;
}

static bool geom_ok(const int dims[4], Geom &g)
{
    for (int k = 0; k < 4; k++)
        if (dims[k] < 2 || dims[k] > kMaxL || (dims[k] % 2)) return false;
    g.T = dims[0];
    g.Lx = dims[1];
    g.Ly = dims[2];
    g.Lz = dims[3];
    g.Lxh = g.Lx / 2;
    g.Lmax = std::max(std::max(g.T, g.Lx), std::max(g.Ly, g.Lz));
    g.V = (long long)g.T * g.Lx * g.Ly * g.Lz;
    g.Vh = g.V / 2;
    return true;
}

}  // namespace dp

using namespace dp;

#define CTX_CHECK(ctx)                                  \
    do {                                                \
        if (!(ctx)) {                                   \
            set_error("null context");                  \
            return DP_ERR_INVALID_ARG;                  \
        }                                               \
        if (cudaSetDevice((ctx)->c.device) != cudaSuccess) { \
            set_error("cudaSetDevice(%d) failed", (ctx)->c.device); \
            return DP_ERR_CUDA;                         \
        }                                               \
    } while (0)

extern "C" {

const char *dp_last_error(void) { return g_err.c_str(); }

dp_status dp_create(dp_ctx **out, int device, const dp_alloc_hooks *hooks, void *stream)
{
    if (!out) {
        set_error("out is null");
        return DP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("no CUDA device %d (%d visible)", device, ndev);
        return DP_ERR_CUDA;
    }
    CUDA_OK(cudaSetDevice(device));
    // a new context may follow a device reset, which invalidates the scratch
    // array's looked-up address of dp_restore_contract_noalloc
    noalloc_forget_address(device);
    dp_ctx *ctx = new dp_ctx();
    Ctx &c = ctx->c;
    c.device = device;
    if (hooks) {
        if (!hooks->alloc || !hooks->free) {
            delete ctx;
            set_error("allocation hooks need both alloc and free");
            return DP_ERR_INVALID_ARG;
        }
        c.hooks = *hooks;
        c.has_hooks = true;
    }
    if (!hooks) {
        cudaMemPoolProps pp{};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = device;
        uint64_t keep = ~0ull;
        if (cudaMemPoolCreate(&c.pool, &pp) != cudaSuccess ||
            cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            if (c.pool) cudaMemPoolDestroy(c.pool);
            delete ctx;
            set_error("cannot create the device memory pool");
            return DP_ERR_CUDA;
        }
    }
    if (stream) {
        c.stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            set_error("cannot create stream");
            return DP_ERR_CUDA;
        }
        c.own_stream = true;
    }
    c.bc.blocks = 2048;
    c.bc.partials = (double *)c.alloc((size_t)c.bc.blocks * kMaxRhs * kRedWidth * sizeof(double));
    c.bc.counter = (unsigned int *)c.alloc(256);
    c.bc.n_active = (int *)c.alloc(256);
    if (!c.bc.partials || !c.bc.counter || !c.bc.n_active ||
        cudaMallocHost(&c.h_nactive, sizeof(int)) != cudaSuccess) {
        dp_destroy(ctx);
        set_error("out of memory creating context");
        return DP_ERR_OOM;
    }
    cudaMemsetAsync(c.bc.counter, 0, 256, c.stream);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) {
        dp_destroy(ctx);
        set_error("stream error creating context");
        return DP_ERR_CUDA;
    }
    *out = ctx;
    return DP_OK;
}

void dp_serve_shutdown(dp_ctx *ctx);

void dp_destroy(dp_ctx *ctx)
{
    if (!ctx) return;
    Ctx &c = ctx->c;
    cudaSetDevice(c.device);
    dp_serve_shutdown(ctx);
    cudaStreamSynchronize(c.stream);
    c.pending.clear();
    std::vector<void *> ps;
    for (auto &kv : c.allocs) ps.push_back(kv.first);
    for (void *p : ps) c.release(p);
    cudaStreamSynchronize(c.stream);
    for (auto e : c.event_pool) cudaEventDestroy(e);
    if (c.h_nactive) cudaFreeHost(c.h_nactive);
    if (c.own_stream) cudaStreamDestroy(c.stream);
    if (c.pool) cudaMemPoolDestroy(c.pool);
    delete ctx;
}

dp_status dp_trim(dp_ctx *ctx)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    if (!c.pool) return DP_OK;
    CUDA_OK(cudaSetDevice(c.device));
    CUDA_OK(cudaStreamSynchronize(c.stream));
    CUDA_OK(cudaMemPoolTrimTo(c.pool, 0));
    return DP_OK;
}

size_t dp_device_bytes(dp_ctx *ctx)
{
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lk(ctx->c.mu);
    return ctx->c.bytes;
}

dp_status dp_field_load(dp_ctx *ctx, const double *links, const int dims[4], int bc_t,
                        dp_field *out)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    if (!links || !dims || !out || (bc_t != 1 && bc_t != -1 && bc_t != 0)) {
        set_error("dp_field_load: null pointer or bc_t not -1, 0 or +1");
        return DP_ERR_INVALID_ARG;
    }
    Geom g;
    if (!geom_ok(dims, g)) {
        set_error("dims must be even and in [2, %d]", kMaxL);
        return DP_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)g.V * 4 * 18;
    for (size_t k = 0; k < n; k++)
        if (!std::isfinite(links[k])) {
            set_error("links contain NaN/Inf at element %zu", k);
            return DP_ERR_INVALID_ARG;
        }
    auto f = std::make_shared<Field>();
    f->g = g;
    f->bc_t = bc_t;
    double2 *lex = (double2 *)c.alloc(n * sizeof(double));
    bool ok = lex != nullptr;
    for (int p = 0; p < 2 && ok; p++) {
        f->l64[p] = (double2 *)c.alloc(g.Vh * 4 * 9 * sizeof(double2));
        f->l32f[p] = (float2 *)c.alloc(g.Vh * 4 * 9 * sizeof(float2));
        f->l32c[p] = (float4 *)c.alloc(g.Vh * 4 * 3 * sizeof(float4));
        ok = f->l64[p] && f->l32f[p] && f->l32c[p];
    }
    if (!ok) {
        c.release(lex);
        for (int p = 0; p < 2; p++) {
            c.release(f->l64[p]);
            c.release(f->l32f[p]);
            c.release(f->l32c[p]);
        }
        set_error("out of device memory loading field");
        return DP_ERR_OOM;
    }
    CUDA_OK(cudaMemcpyAsync(lex, links, n * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    CUDA_OK(launch_pack_links(lex, g, f->l64, f->l32f, f->l32c, c.stream));
    c.launches++;
    CUDA_OK(cudaStreamSynchronize(c.stream));
    c.release(lex);
    std::lock_guard<std::mutex> lk(c.mu);
    const uint64_t id = c.next_field++;
    c.fields[id] = f;
    *out = id;
    return DP_OK;
}

dp_status dp_field_set_csw(dp_ctx *ctx, dp_field field, double csw)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    auto f = find_field(&c, field);
    if (!f) {
        set_error("unknown field %llu", (unsigned long long)field);
        return DP_ERR_NOT_FOUND;
    }
    if (!std::isfinite(csw)) {
        set_error("c_sw is not finite");
        return DP_ERR_INVALID_ARG;
    }
    const long long Vh = f->g.Vh;
    for (int p = 0; p < 2; p++) {
        if (!f->clov[p]) f->clov[p] = (double2 *)c.alloc(Vh * 36 * sizeof(double2));
        if (!f->clov32[p]) f->clov32[p] = (float4 *)c.alloc(Vh * 18 * sizeof(float4));
        if (!f->clov[p] || !f->clov32[p]) {
            set_error("out of device memory (clover)");
            return DP_ERR_OOM;
        }
    }
    CUDA_OK(launch_clover_build(f->l64[0], f->l64[1], f->g, csw, f->clov[0], f->clov[1], c.stream));
    c.launches++;
    // FP32 copy of the clover term for the FP32 apply path
    for (int p = 0; p < 2; p++) CUDA_OK(launch_clover_to_f32(f->clov[p], f->clov32[p], Vh, c.stream));
    c.launches += 2;
    CUDA_OK(cudaStreamSynchronize(c.stream));
    {
        std::lock_guard<std::mutex> lk(f->inv_mu);
        f->invs.clear();
    }
    f->has_clover = true;
    f->csw = csw;
    return DP_OK;
}

dp_status dp_field_free(dp_ctx *ctx, dp_field field)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    std::shared_ptr<Field> f;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.fields.find(field);
        if (it == c.fields.end()) {
            set_error("unknown field %llu", (unsigned long long)field);
            return DP_ERR_NOT_FOUND;
        }
        if (it->second->users.load() > 0) {
            set_error("field has requests in flight");
            return DP_ERR_INVALID_ARG;
        }
        f = it->second;
        c.fields.erase(it);
    }
    cudaStreamSynchronize(c.stream);
    for (int p = 0; p < 2; p++) {
        c.release(f->l64[p]);
        c.release(f->l32f[p]);
        c.release(f->l32c[p]);
        c.release(f->clov[p]);
        c.release(f->clov32[p]);
        c.release(f->l16[0][p]);
        c.release(f->l16[1][p]);
        c.release(f->ldf[p]);
    }
    {
        std::lock_guard<std::mutex> lk(f->inv_mu);
        f->invs.clear();
    }
    cudaStreamSynchronize(c.stream);
    return DP_OK;
}

dp_status dp_apply(dp_ctx *ctx, dp_field field, int kind, double M, const dp_profile *profile,
                   const int src[4], int prec, int compress12, const double *in, double *out,
                   int nrhs)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    Field &f = *fp;
    if (!in || !out || nrhs < 1 || nrhs > kMaxRhs || kind < 0 || kind > 3 || prec < DP_PREC_FP64 ||
        prec > DP_PREC_MIXED_BF16 || !std::isfinite(M)) {
        set_error("dp_apply: invalid argument");
        return DP_ERR_INVALID_ARG;
    }
    if (kind != DP_APPLY_HOP && !f.has_clover) {
        set_error("clover term not built");
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = f.g;
    const size_t nlex = (size_t)g.V * 24 * nrhs;
    for (size_t k = 0; k < nlex; k++)
        if (!std::isfinite(in[k])) {
            set_error("input spinor has NaN/Inf");
            return DP_ERR_INVALID_ARG;
        }
    const int pr = prec == DP_PREC_FP64 ? 0 : 1;
    const int zero_src[4] = {0, 0, 0, 0};
    dp_profile none{};
    none.kind = DP_PROF_NONE;
    std::vector<double> alpha(4 * g.Lmax), hop(8 * g.Lmax);
    dp_status stt = profile_tables(profile ? *profile : none, g, f.bc_t, src ? src : zero_src,
                                   alpha.data(), hop.data());
    if (stt != DP_OK) return stt;
    std::vector<float> hopf(hop.begin(), hop.end());
    const int lf = inner_link_format(prec, compress12);
    const void *links[2];
    for (int p = 0; p < 2; p++) {
        stt = field_links(&c, f, lf, p, &links[p]);
        if (stt != DP_OK) return stt;
    }

    std::shared_ptr<CloverInv> ci;
    if (kind == DP_APPLY_CLOVER_INV) {
        stt = get_clover_inv(&c, f, M, &ci);
        if (stt != DP_OK) return stt;
    }
    // FP32 kernels work on RHS pairs: an odd count gets one zero RHS appended
    const int nk = (pr == 1 && (nrhs & 1)) ? nrhs + 1 : nrhs;
    const size_t nlex_k = (size_t)g.V * 24 * nk;
    const size_t vb = (size_t)g.Vh * nk * 24 * (pr == 0 ? 8 : 4);
    double2 *lex = (double2 *)c.alloc(nlex_k * sizeof(double));
    void *ie = c.alloc(vb), *io = c.alloc(vb), *oe = c.alloc(vb), *oo = c.alloc(vb);
    void *te = c.alloc(vb), *to = c.alloc(vb);
    void *hopd = c.alloc(hop.size() * sizeof(double));
    dp_status ret = DP_OK;
    if (!lex || !ie || !io || !oe || !oo || !te || !to || !hopd) {
        set_error("out of device memory (dp_apply)");
        ret = DP_ERR_OOM;
    } else {
        auto run = [&]() -> dp_status {
            if (nk > nrhs)
                CUDA_OK(cudaMemsetAsync((double *)lex + nlex, 0, (nlex_k - nlex) * sizeof(double), c.stream));
            CUDA_OK(cudaMemcpyAsync(lex, in, nlex * sizeof(double), cudaMemcpyHostToDevice, c.stream));
            CUDA_OK(launch_pack_spinor(lex, g, nk, pr, ie, io, c.stream));
            if (pr == 0)
                CUDA_OK(cudaMemcpyAsync(hopd, hop.data(), hop.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, c.stream));
            else
                CUDA_OK(cudaMemcpyAsync(hopd, hopf.data(), hopf.size() * sizeof(float),
                                        cudaMemcpyHostToDevice, c.stream));
            void *inp[2] = {ie, io}, *outp[2] = {oe, oo}, *tmp[2] = {te, to};
            for (int p = 0; p < 2; p++) {
                const void *mat;
                if (kind == DP_APPLY_CLOVER_INV)
                    mat = pr == 0 ? (const void *)ci->inv64[p] : (const void *)ci->inv32[p];
                else
                    mat = pr == 0 ? (const void *)f.clov[p] : (const void *)f.clov32[p];
                CloverApplyParams cp{};
                cp.mat[0] = mat;
                cp.diag[0] = kind == DP_APPLY_FULL ? 4.0 + M : 0.0;
                cp.Vh = g.Vh;
                cp.nrhs = nk;
                cp.in = inp[p];
                cp.out = (kind == DP_APPLY_FULL) ? tmp[p] : outp[p];
                if (kind == DP_APPLY_CLOVER || kind == DP_APPLY_CLOVER_INV) {
                    CUDA_OK(launch_clover_apply(cp, pr, c.stream));
                    continue;
                }
                DslashParams P{};
                P.in = inp[1 - p];
                P.out = outp[p];
                P.links[0] = links[0];
                P.links[1] = links[1];
                P.hop = hopd;
                P.g = g;
                P.parity = p;
                P.nrhs = nk;
                int epi = EPI_HOP;
                if (kind == DP_APPLY_FULL) {
                    CUDA_OK(launch_clover_apply(cp, pr, c.stream));
                    P.x = tmp[p];
                    epi = EPI_XPY;
                }
                const Shape sh = c.launch_shape(g.Vh, pr, lf, nk);
                CUDA_OK(launch_dslash(P, pr, lf, epi, sh.block, pr == 0 ? 1 : 2, c.stream));
            }
            CUDA_OK(launch_unpack_spinor(oe, oo, g, nk, pr, lex, c.stream));
            CUDA_OK(cudaMemcpyAsync(out, lex, nlex * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
            CUDA_OK(cudaStreamSynchronize(c.stream));
            c.launches += 6;
            return DP_OK;
        };
        ret = run();
    }
    c.release(lex);
    c.release(ie);
    c.release(io);
    c.release(oe);
    c.release(oo);
    c.release(te);
    c.release(to);
    c.release(hopd);
    cudaStreamSynchronize(c.stream);
    return ret;
}

size_t dp_spinor_bytes(dp_ctx *ctx, dp_field field, int prec, int nrhs)
{
    if (!ctx) return 0;
    auto f = find_field(&ctx->c, field);
    if (!f) return 0;
    return (size_t)f->g.Vh * nrhs * 24 * (prec == DP_PREC_FP64 ? 8 : 4);
}

dp_status dp_dslash_dev(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                        int prec, int compress12, int out_parity, const void *in, void *out,
                        int nrhs, int block_threads, int rhs_per_thread, int stages, int iters,
                        float *ms_out)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    Field &f = *fp;
    if (!in || !out || nrhs < 1 || nrhs > kMaxRhs || iters < 1 || (out_parity & ~1) ||
        prec < DP_PREC_FP64 || prec > DP_PREC_MIXED_BF16 ||
        rhs_per_thread < 0 || stages < -1 || stages > 6 ||
        (block_threads != 0 && (block_threads < 32 || block_threads > 256 || block_threads % 32))) {
        set_error("dp_dslash_dev: invalid argument");
        return DP_ERR_INVALID_ARG;
    }
    const int want_rpt = rhs_per_thread;
    if (rhs_per_thread != 0 &&
        !dslash_rpt_ok(nrhs, want_rpt, prec == DP_PREC_FP64 ? 0 : 1, EPI_AINV)) {
        set_error("dp_dslash_dev: launch shape %d is not available for %d RHS in this precision",
                  rhs_per_thread, nrhs);
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = f.g;
    const int pr = prec == DP_PREC_FP64 ? 0 : 1;
    const int lf = inner_link_format(prec, compress12);
    const void *links[2];
    for (int p = 0; p < 2; p++) {
        dp_status s2 = field_links(&c, f, lf, p, &links[p]);
        if (s2 != DP_OK) return s2;
    }
    std::shared_ptr<CloverInv> ci;
    dp_status stt = get_clover_inv(&c, f, M, &ci);
    if (stt != DP_OK) return stt;
    const int zero_src[4] = {0, 0, 0, 0};
    dp_profile none{};
    none.kind = DP_PROF_NONE;
    std::vector<double> alpha(4 * g.Lmax), hop(8 * g.Lmax);
    stt = profile_tables(profile ? *profile : none, g, f.bc_t, zero_src, alpha.data(), hop.data());
    if (stt != DP_OK) return stt;
    std::vector<float> hopf(hop.begin(), hop.end());
    void *hopd = c.alloc(hop.size() * sizeof(double));
    if (!hopd) {
        set_error("out of device memory");
        return DP_ERR_OOM;
    }
    if (pr == 0)
        CUDA_OK(cudaMemcpyAsync(hopd, hop.data(), hop.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    else
        CUDA_OK(cudaMemcpyAsync(hopd, hopf.data(), hopf.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    DslashParams P{};
    P.in = in;
    P.out = out;
    P.links[0] = links[0];
    P.links[1] = links[1];
    P.clov[0] = pr == 0 ? (const void *)ci->inv64[out_parity] : (const void *)ci->inv32[out_parity];
    P.hop = hopd;
    P.g = g;
    P.parity = out_parity;
    P.nrhs = nrhs;
    const Shape sh = c.launch_shape(g.Vh, pr, lf, nrhs);
    int block = sh.block, rpt = sh.rpt, stg = sh.stages;
    if (block_threads > 0) block = block_threads;
    if (rhs_per_thread != 0) rpt = want_rpt;
    if (stages >= 0) stg = stages;
    if (stg > 0 && !dslash_staged_ok(pr, lf, EPI_AINV, rpt, stg, block)) {
        c.release(hopd);
        set_error("dp_dslash_dev: shared-memory staging needs FP32 or 16-bit 12-real links, 2 RHS per "
                  "thread and 64, 96 or 128 threads per block");
        return DP_ERR_INVALID_ARG;
    }
    cudaEvent_t a = c.get_event(), b = c.get_event();
    CUDA_OK(cudaEventRecord(a, c.stream));
    for (int k = 0; k < iters; k++)
        CUDA_OK(launch_dslash(P, pr, lf, EPI_AINV, block, rpt, c.stream, stg));
    CUDA_OK(cudaEventRecord(b, c.stream));
    c.launches += iters;
    CUDA_OK(cudaEventSynchronize(b));
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    c.event_pool.push_back(a);
    c.event_pool.push_back(b);
    if (ms_out) *ms_out = ms / iters;
    c.release(hopd);
    return DP_OK;
}

dp_status dp_autotune(dp_ctx *ctx, dp_field field, int prec, int compress12, int nrhs,
                      int *best_block_threads, int *best_rhs_per_thread, int *best_stages,
                      float *best_ms)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    if (nrhs < 1 || nrhs > kMaxRhs || prec < DP_PREC_FP64 || prec > DP_PREC_MIXED_BF16) {
        set_error("dp_autotune: invalid argument");
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = fp->g;
    const int pr = prec == DP_PREC_FP64 ? 0 : 1;
    const int lf = inner_link_format(prec, compress12);
    const size_t vb = dp_spinor_bytes(ctx, field, prec, nrhs);
    void *in = c.alloc(vb), *out = c.alloc(vb);
    if (!in || !out) {
        c.release(in);
        c.release(out);
        set_error("out of device memory (autotune)");
        return DP_ERR_OOM;
    }
    cudaMemsetAsync(in, 0, vb, c.stream);
    // candidates: four block sizes x RHS per thread (FP64: 1; FP32: one or
    // two RHS pairs) x how neighbour data arrives (FP32 one pair per thread:
    // direct, shared-memory staging of spinor and link 2-3 directions ahead
    // or in a persistent wave, direct with an L1 prefetch 2 directions ahead,
    // or the spinor alone staged 2 directions ahead with the link from L1)
    const int blocks[] = {64, 96, 128, 192, 256};
    const int rpts[] = {1, 2, 4};
    const int stage_opts[] = {0, 2, 3, 4, 5, 6};
    Shape best;
    float bms = 1e30f;
    dp_status st = DP_OK;
    for (int r : rpts) {
        if (!dslash_rpt_ok(nrhs, r, pr, EPI_AINV)) continue;
        for (int sg : stage_opts) {
            for (int b : blocks) {
                if (sg > 0 && !dslash_staged_ok(pr, lf, EPI_AINV, r, sg, b)) continue;
                float ms = 0;
                // warm up once, then time a few launches
                st = dp_dslash_dev(ctx, field, 0.1, nullptr, prec, compress12, 0, in, out, nrhs, b,
                                   r, sg, 2, &ms);
                if (st != DP_OK) break;
                st = dp_dslash_dev(ctx, field, 0.1, nullptr, prec, compress12, 0, in, out, nrhs, b,
                                   r, sg, 10, &ms);
                if (st != DP_OK) break;
                if (ms < bms) {
                    bms = ms;
                    best.block = b;
                    best.rpt = r;
                    best.stages = sg;
                }
            }
            if (st != DP_OK) break;
        }
        if (st != DP_OK) break;
    }
    c.release(in);
    c.release(out);
    if (st != DP_OK) return st;
    if (bms >= 1e30f) {
        set_error("dp_autotune: no launch shape serves %d RHS in this precision (FP32 needs an even count)", nrhs);
        return DP_ERR_INVALID_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(c.mu);
        c.tuned[TuneKey{g.Vh, pr, lf, nrhs}] = best;
    }
    if (best_block_threads) *best_block_threads = best.block;
    if (best_rhs_per_thread) *best_rhs_per_thread = best.rpt;
    if (best_stages) *best_stages = best.stages;
    if (best_ms) *best_ms = bms;
    return DP_OK;
}

dp_status dp_tune_set(dp_ctx *ctx, dp_field field, int prec, int compress12, int nrhs,
                      int block_threads, int rhs_per_thread, int stages)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    if (nrhs < 1 || nrhs > kMaxRhs || prec < DP_PREC_FP64 || prec > DP_PREC_MIXED_BF16) {
        set_error("dp_tune_set: invalid argument");
        return DP_ERR_INVALID_ARG;
    }
    const int pr = prec == DP_PREC_FP64 ? 0 : 1;
    const int lf = inner_link_format(prec, compress12);
    const bool ok = block_threads > 0 && block_threads <= 256 && block_threads % 32 == 0 &&
                    dslash_rpt_ok(nrhs, rhs_per_thread, pr, EPI_AINV) &&
                    dslash_rpt_ok(nrhs, rhs_per_thread, pr, EPI_XMY_AINV) &&
                    (stages == 0 || (dslash_staged_ok(pr, lf, EPI_AINV, rhs_per_thread, stages, block_threads) &&
                                     dslash_staged_ok(pr, lf, EPI_XMY_AINV, rhs_per_thread, stages,
                                                      block_threads)));
    if (!ok) {
        set_error("dp_tune_set: shape (%d threads, %d RHS per thread, stages %d) cannot serve %d RHS here",
                  block_threads, rhs_per_thread, stages, nrhs);
        return DP_ERR_INVALID_ARG;
    }
    Shape sh;
    sh.block = block_threads;
    sh.rpt = rhs_per_thread;
    sh.stages = stages;
    std::lock_guard<std::mutex> lk(c.mu);
    c.tuned[TuneKey{fp->g.Vh, pr, lf, nrhs}] = sh;
    return DP_OK;
}

dp_status dp_timing_enable(dp_ctx *ctx, int on)
{
    CTX_CHECK(ctx);
    ctx->c.timing = on != 0;
    return DP_OK;
}

dp_status dp_timing_reset(dp_ctx *ctx)
{
    CTX_CHECK(ctx);
    ctx->c.collect_timing();
    ctx->c.stats.clear();
    return DP_OK;
}

dp_status dp_timing_get(dp_ctx *ctx, const char *name, long *launches, double *total_ms)
{
    CTX_CHECK(ctx);
    if (!name) {
        set_error("null name");
        return DP_ERR_INVALID_ARG;
    }
    ctx->c.collect_timing();
    auto it = ctx->c.stats.find(name);
    if (launches) *launches = it == ctx->c.stats.end() ? 0 : it->second.launches;
    if (total_ms) *total_ms = it == ctx->c.stats.end() ? 0 : it->second.ms;
    return DP_OK;
}

long dp_launch_count(dp_ctx *ctx) { return ctx ? ctx->c.launches.load() : 0; }

dp_status dp_restore_contract_dev(dp_ctx *ctx, dp_field field, int n_groups,
                                  const dp_profile *profiles, const int *src, const double *xe,
                                  const double *xo, double *cpp_dev)
{
    CTX_CHECK(ctx);
    Ctx &c = ctx->c;
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    if (n_groups < 1 || n_groups > kMaxGroups || 12 * n_groups > kMaxRhs || !profiles || !src ||
        !xe || !xo || !cpp_dev) {
        set_error("dp_restore_contract_dev: invalid argument (n_groups in [1, %d])", kMaxRhs / 12);
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = fp->g;
    const int Lm = g.Lmax, n = 12 * n_groups;
    const int L[4] = {g.T, g.Lx, g.Ly, g.Lz};
    std::vector<double> alpha((size_t)n_groups * 4 * Lm), hop(8 * Lm);
    std::vector<SlotInfo> slots(n);
    std::vector<int> tsrc(n_groups);
    for (int k = 0; k < n_groups; k++) {
        for (int mu = 0; mu < 4; mu++)
            if (src[4 * k + mu] < 0 || src[4 * k + mu] >= L[mu]) {
                set_error("source coordinate out of range");
                return DP_ERR_INVALID_ARG;
            }
        dp_status s = profile_tables(profiles[k], g, fp->bc_t, src + 4 * k,
                                     &alpha[(size_t)k * 4 * Lm], hop.data());
        if (s != DP_OK) return s;
        tsrc[k] = src[4 * k];
        for (int j = 0; j < 12; j++) {
            SlotInfo &sl = slots[12 * k + j];
            sl.group = k;
            sl.comp = j;
            sl.t = src[4 * k];
            sl.x = src[4 * k + 1];
            sl.y = src[4 * k + 2];
            sl.z = src[4 * k + 3];
            sl.scale = 1.0;
        }
    }
    const size_t npart = (size_t)g.T * contract_blocks_per_slice(g) * n_groups;
    double *alpha_d = (double *)c.alloc(alpha.size() * sizeof(double));
    SlotInfo *slots_d = (SlotInfo *)c.alloc(sizeof(SlotInfo) * n);
    int *tsrc_d = (int *)c.alloc(sizeof(int) * n_groups);
    double *part = (double *)c.alloc(npart * sizeof(double));
    dp_status ret = DP_OK;
    if (!alpha_d || !slots_d || !tsrc_d || !part) {
        set_error("out of device memory (restore/contract scratch)");
        ret = DP_ERR_OOM;
    } else {
        cudaError_t e = cudaMemcpyAsync(alpha_d, alpha.data(), alpha.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slots_d, slots.data(), sizeof(SlotInfo) * n, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tsrc_d, tsrc.data(), sizeof(int) * n_groups, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess)
            e = launch_restore_contract((const double2 *)xe, (const double2 *)xo, g, n, alpha_d, slots_d,
                                        n_groups, tsrc_d, nullptr, cpp_dev, part, nullptr, c.stream);
        // the host tables are pageable: make sure the copies are done before they go
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) {
            set_error("restore/contract: %s", cudaGetErrorString(e));
            ret = DP_ERR_CUDA;
        }
        c.launches += 2;
    }
    c.release(alpha_d);
    c.release(slots_d);
    c.release(tsrc_d);
    c.release(part);
    return ret;
}

dp_status dp_profile_tables(const int dims[4], int bc_t, const dp_profile *profile,
                            const int src[4], double *alpha_out, double *hop_out)
{
    if (!dims || !profile || !alpha_out || !hop_out || (bc_t != 1 && bc_t != -1 && bc_t != 0)) {
        set_error("dp_profile_tables: invalid argument");
        return DP_ERR_INVALID_ARG;
    }
    Geom g;
    if (!geom_ok(dims, g)) {
        set_error("dims must be even and in [2, %d]", kMaxL);
        return DP_ERR_INVALID_ARG;
    }
    const int zero[4] = {0, 0, 0, 0};
    const int *s = src ? src : zero;
    const int L[4] = {g.T, g.Lx, g.Ly, g.Lz};
    for (int mu = 0; mu < 4; mu++)
        if (s[mu] < 0 || s[mu] >= L[mu]) {
            set_error("source coordinate out of range");
            return DP_ERR_INVALID_ARG;
        }
    return profile_tables(*profile, g, bc_t, s, alpha_out, hop_out);
}

}  // extern "C"
