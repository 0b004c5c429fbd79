// C-ABI layer of liblbm (declared in include/lbm.h): handle management,
// parameter checks, host-side constants of the step, and launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_internal.h"

using lbm::Geometry;
using lbm::StepConst;

struct lbm_ctx {
    int nx = 0, ny = 0;
    int storage = 0;
    int bc = 0;
    int device = 0;
    double rho0 = 1, ux0 = 0, uy0 = 0;
    lbm_rates rates{};
    cudaStream_t stream = nullptr;
    lbm_allocator alloc{};
    bool custom_alloc = false;
    Geometry geo{};
    size_t buf_bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;  // buffer holding the post-collision state the next pull reads
    void* chi_x = nullptr;  // device AxisCoef tables (chi, 1/(1+n chi), 1/(1+m chi)), compute precision
    void* chi_y = nullptr;
    size_t chi_bytes_x = 0, chi_bytes_y = 0;
    double* diag = nullptr;  // kDiagBlocks * kDiag partials followed by kDiag results
    size_t diag_bytes = 0;
    double* staging = nullptr;  // 3 FP64 fields for host transfers, allocated on first use
    size_t staging_bytes = 0;
    int variant = 0;
    double rho_f = 1, ux_f = 0, uy_f = 0;
    int bulk[4] = {0, 0, 0, 0};  // rectangle [x0, x1) x [y0, y1) where chi = 0
    StepConst<double> k64{};
    StepConst<float> k32{};
    StepConst<lbm::F2> k2{};          // the FP32 constants, duplicated for the pair kernel
    StepConst<lbm::FF> kff{};         // float-float constants of the compensated step
    int arith = LBM_ARITH_NATIVE;     // LBM_ARITH_COMPENSATED: FP32 storage, float-float collision
    int cpt = 1;                      // cells per thread of the step kernel: 1, or 2 (FP32 / 16-bit)
    int spl = 1;                      // time steps per launch: 1, or 2 (needs cpt == 2)
    lbm::LineSource src{};            // channel boundary: the line source (amp 0 until lbm_set_source)
    long long* d_time = nullptr;      // channel boundary: device copy of the step counter
    double* d_src_table = nullptr;    // channel boundary: source scales of the next kGraphChunk steps,
                                      // then their FP32 source populations (9 per step)
    bool initialised = false;
    int64_t time = 0;
    int launch_mode = 2;              // kLaunchGraph; LBM_LAUNCH=plain|pdl|graph overrides
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // kGraphChunk steps from buffer 0 / 1
    bool tma = false;                 // two-step launches stage their input by TMA (FP32, Dirichlet)
    bool tma_ready = false;           // tmap / tma_grid / tma_err are set up
    CUtensorMap tmap[2];              // tensor maps of buf[0], buf[1]
    int tma_grid = 0;                 // persistent CTAs of the TMA kernel
    int* tma_err = nullptr;           // set on the device when a staged copy timed out
    int tma_polls = -1;               // polls of each staged copy's wait (< 0: default)
    cudaStream_t capture_stream = nullptr;
    std::string err;
};

namespace {

// How lbm_step issues its kernels: one launch per step; one launch per step as
// a programmatic dependent of the previous (its launch overlaps the previous
// step's tail); or replays of a captured graph of kGraphChunk such launches.
enum { kLaunchPlain = 0, kLaunchPdl = 1, kLaunchGraph = 2 };
constexpr int kGraphChunk = 64;  // even, so a replay returns to the same buffer

thread_local std::string g_create_error;

int fail(lbm_ctx* h, int code, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(lbm_ctx* h, cudaError_t e, const char* where) {
    return fail(h, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(lbm_ctx* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (h->custom_alloc) return h->alloc.alloc(bytes, h->alloc.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_ctx* h, void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (h->custom_alloc)
        h->alloc.free(p, bytes, h->alloc.ctx);
    else
        cudaFree(p);
}

// Make the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

template <typename CT>
void fill_const(const lbm_ctx* h, StepConst<CT>& k) {
    k = lbm::make_step_const<CT>(h->rates.s, h->rates.n, h->rates.m, h->rho0, h->ux0, h->uy0,
                                 h->rho_f, h->ux_f, h->uy_f, h->bulk);
}

void refresh_consts(lbm_ctx* h) {
    fill_const<double>(h, h->k64);
    fill_const<float>(h, h->k32);
    fill_const<lbm::F2>(h, h->k2);
    fill_const<lbm::FF>(h, h->kff);
}

int ensure_staging(lbm_ctx* h) {
    const size_t need = 3 * sizeof(double) * (size_t)h->nx * h->ny;
    if (h->staging && h->staging_bytes >= need) return LBM_OK;
    dev_free(h, h->staging, h->staging_bytes);
    h->staging = static_cast<double*>(dev_alloc(h, need));
    h->staging_bytes = h->staging ? need : 0;
    if (!h->staging) return fail(h, LBM_ERR_OOM, "staging allocation failed");
    return LBM_OK;
}

// e_i = f^eq_i(1, u0) of the line source (channel boundary), in FP64.
void set_source_shape(lbm_ctx* h) {
    const double ux = h->ux0, uy = h->uy0, uu = ux * ux + uy * uy;
    const int CXS[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int CYS[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int i = 0; i < 9; ++i) {
        const double cu = CXS[i] * ux + CYS[i] * uy;
        h->src.e[i] = W[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

// The pair kernel steps FP32 and 16-bit storage and addresses the nine
// planes with 32-bit element offsets.
bool pair_kernel_ok(const lbm_ctx* h) {
    return h->storage != LBM_F64 && 9 * h->geo.plane < (1ll << 32);
}

lbm::BaseState base_of(const lbm_ctx* h) { return lbm::BaseState{h->rho0, h->ux0, h->uy0}; }

bool is_finite(double v) { return std::isfinite(v); }

// The line source as a step launch sees it: the device step counter plus
// t_off launches issued since it was last advanced.
// The line source as the step kernels see it: the scale of step t_off of the
// current chunk, from the table source_table_kernel filled at its start.
lbm::LineSource launch_source(const lbm_ctx* h, long long t_off) {
    lbm::LineSource ls = h->src;
    ls.time = h->d_time;
    ls.t_off = t_off;
    ls.table = h->d_src_table;
    ls.pop = h->d_src_table ? reinterpret_cast<const float*>(h->d_src_table + kGraphChunk) : nullptr;
    return ls;
}

// The line source as the read-out kernels see it: the state of time h->time.
lbm::LineSource readout_source(const lbm_ctx* h) {
    lbm::LineSource ls = h->src;
    ls.time = nullptr;
    ls.t_off = h->time;
    ls.table = nullptr;
    ls.pop = nullptr;
    return ls;
}

__global__ void advance_time_kernel(long long* t, int by) { *t += by; }

// table[k] = the source scale of step k of the chunk starting at the device
// clock, k < n, and pop[9 k + i] = float(table[k] e_i) its FP32 source
// populations: the FP64 sine and products evaluated once per step here
// instead of in the edge threads of every step kernel (on the critical path
// of each launch).
__global__ void source_table_kernel(const long long* time, double* table, float* pop, int n,
                                    lbm::LineSource ls) {
    const int k = threadIdx.x;
    if (k >= n) return;
    ls.time = time;
    ls.t_off = k;
    ls.table = nullptr;
    const double scale = lbm::line_source_scale(ls);
    table[k] = scale;
    for (int i = 0; i < 9; ++i) pop[9 * k + i] = static_cast<float>(scale * ls.e[i]);
}

// Fill the table for the next n <= kGraphChunk steps (channel boundary only).
cudaError_t launch_source_table(lbm_ctx* h, cudaStream_t st, int n) {
    source_table_kernel<<<1, kGraphChunk, 0, st>>>(
        h->d_time, h->d_src_table, reinterpret_cast<float*>(h->d_src_table + kGraphChunk), n,
        h->src);
    return cudaGetLastError();
}

cudaError_t launch_one_step(lbm_ctx* h, const void* src, void* dst, cudaStream_t st, bool pdl,
                            long long t_off = 0) {
    const int p = pdl ? 1 : 0;
    const lbm::LineSource ls = launch_source(h, t_off);
    const auto* tx = static_cast<const lbm::AxisCoef<float>*>(h->chi_x);
    const auto* ty = static_cast<const lbm::AxisCoef<float>*>(h->chi_y);
    if (h->arith == LBM_ARITH_COMPENSATED)
        return lbm::launch_step_ff(src, dst, h->geo, h->kff, tx, ty, h->variant, h->bc, st, p, ls);
    if (h->cpt == 2) {
        switch (h->storage) {
            case LBM_F32: return lbm::launch_step2_f32(src, dst, h->geo, h->k2, tx, ty, h->variant, h->bc, st, p, ls);
            case LBM_F16DEV: return lbm::launch_step2_f16(src, dst, h->geo, h->k2, tx, ty, h->variant, h->bc, st, p, ls);
            case LBM_BF16DEV: return lbm::launch_step2_bf16(src, dst, h->geo, h->k2, tx, ty, h->variant, h->bc, st, p, ls);
            default: break;
        }
    }
    switch (h->storage) {
        case LBM_F64:
            return lbm::launch_step_f64(src, dst, h->geo, h->k64, static_cast<const lbm::AxisCoef<double>*>(h->chi_x),
                                        static_cast<const lbm::AxisCoef<double>*>(h->chi_y), h->variant, h->bc, st, p, ls);
        case LBM_F32:
            return lbm::launch_step_f32(src, dst, h->geo, h->k32, static_cast<const lbm::AxisCoef<float>*>(h->chi_x),
                                        static_cast<const lbm::AxisCoef<float>*>(h->chi_y), h->variant, h->bc, st, p, ls);
        case LBM_F16DEV:
            return lbm::launch_step_f16(src, dst, h->geo, h->k32, static_cast<const lbm::AxisCoef<float>*>(h->chi_x),
                                        static_cast<const lbm::AxisCoef<float>*>(h->chi_y), h->variant, h->bc, st, p, ls);
        default:
            return lbm::launch_step_bf16(src, dst, h->geo, h->k32, static_cast<const lbm::AxisCoef<float>*>(h->chi_x),
                                         static_cast<const lbm::AxisCoef<float>*>(h->chi_y), h->variant, h->bc, st, p, ls);
    }
}

// Two steps src (time t) -> dst (time t + 2) in one launch.
cudaError_t launch_two_steps(lbm_ctx* h, const void* src, void* dst, cudaStream_t st, bool pdl) {
    const int p = pdl ? 1 : 0;
    const auto* tx = static_cast<const lbm::AxisCoef<float>*>(h->chi_x);
    const auto* ty = static_cast<const lbm::AxisCoef<float>*>(h->chi_y);
    if (h->tma) {
        const CUtensorMap& m = h->tmap[src == h->buf[0] ? 0 : 1];
        switch (h->storage) {
            case LBM_F32:
                return lbm::launch_step_tb2_tma_f32(m, dst, h->geo, h->k2, tx, ty, h->variant,
                                                    h->tma_grid, h->tma_err, st, p, h->tma_polls);
            case LBM_F16DEV:
                return lbm::launch_step_tb2_tma_f16(m, dst, h->geo, h->k2, tx, ty, h->variant,
                                                    h->tma_grid, h->tma_err, st, p, h->tma_polls);
            case LBM_BF16DEV:
                return lbm::launch_step_tb2_tma_bf16(m, dst, h->geo, h->k2, tx, ty, h->variant,
                                                     h->tma_grid, h->tma_err, st, p, h->tma_polls);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (h->storage) {
        case LBM_F32: return lbm::launch_step_tb2_f32(src, dst, h->geo, h->k2, tx, ty, h->variant, h->bc, st, p);
        case LBM_F16DEV: return lbm::launch_step_tb2_f16(src, dst, h->geo, h->k2, tx, ty, h->variant, h->bc, st, p);
        case LBM_BF16DEV: return lbm::launch_step_tb2_bf16(src, dst, h->geo, h->k2, tx, ty, h->variant, h->bc, st, p);
        default: return cudaErrorInvalidValue;
    }
}

// Tensor maps, persistent grid and error flag of the TMA two-step kernel;
// LBM_OK, or the reason it is not available for this handle.
int setup_tma(lbm_ctx* h) {
    if (h->tma_ready) return LBM_OK;
    if (h->storage == LBM_F64 || h->bc != LBM_BC_DIRICHLET_EQ)
        return fail(h, LBM_ERR_ARG,
                    "TMA staging needs FP32, FP16 or BF16 storage and the Dirichlet boundary");
    int per_sm = 0, sms = 0;
    cudaError_t e = h->storage == LBM_F32      ? lbm::prepare_step_tb2_tma_f32(&per_sm)
                    : h->storage == LBM_F16DEV ? lbm::prepare_step_tb2_tma_f16(&per_sm)
                                               : lbm::prepare_step_tb2_tma_bf16(&per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "TMA kernel set-up");
    if (per_sm < 1) return fail(h, LBM_ERR_CUDA, "the TMA kernel does not fit an SM");
    const int elem = h->storage == LBM_F32 ? 4 : 2;
    const bool bf16 = h->storage == LBM_BF16DEV;
    if (!lbm::encode_tma_map(&h->tmap[0], h->buf[0], h->geo, elem, bf16) ||
        !lbm::encode_tma_map(&h->tmap[1], h->buf[1], h->geo, elem, bf16))
        return fail(h, LBM_ERR_CUDA, "the driver did not encode the tensor maps");
    if (!h->tma_err) {
        h->tma_err = static_cast<int*>(dev_alloc(h, 256));
        if (!h->tma_err) return fail(h, LBM_ERR_OOM, "TMA error flag allocation failed");
        e = cudaMemsetAsync(h->tma_err, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "TMA error flag");
    }
    h->tma_grid = per_sm * sms;
    h->tma_polls = lbm::tma_wait_polls();
    h->tma_ready = true;
    return LBM_OK;
}

// After the stream is synchronised: LBM_ERR_CUDA if a staged copy timed out.
int check_tma(lbm_ctx* h) {
    if (!h->tma_err) return LBM_OK;
    int flag = 0;
    const cudaError_t e = cudaMemcpy(&flag, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "TMA error flag");
    if (flag) return fail(h, LBM_ERR_CUDA, "a TMA-staged copy did not complete within its wait");
    return LBM_OK;
}

void drop_graphs(lbm_ctx* h) {
    for (int i = 0; i < 2; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        h->graph[i] = nullptr;
    }
}

// Capture kGraphChunk consecutive steps starting from buffer `parity` on the
// handle's private capture stream (programmatic dependent launches between
// them) and instantiate the graph; it is replayed on the handle's stream.
cudaError_t ensure_graph(lbm_ctx* h, int parity) {
    if (h->graph[parity]) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!h->capture_stream) {
        e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    if (h->bc == LBM_BC_CHANNEL) e = launch_source_table(h, h->capture_stream, kGraphChunk);
    int c = parity;
    for (int t = 0; t < kGraphChunk && e == cudaSuccess; t += h->spl) {
        if (h->spl == 2)
            e = launch_two_steps(h, h->buf[c], h->buf[1 - c], h->capture_stream, t > 0);
        else
            e = launch_one_step(h, h->buf[c], h->buf[1 - c], h->capture_stream, t > 0, t);
        c = 1 - c;
    }
    if (e == cudaSuccess && h->bc == LBM_BC_CHANNEL) {  // the line source's clock
        advance_time_kernel<<<1, 1, 0, h->capture_stream>>>(h->d_time, kGraphChunk);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" {

const char* lbm_version(void) { return "liblbm 0.1 (D2Q9 MRT + absorbing layers, sm_103a)"; }

size_t lbm_lattice_bytes(int nx, int ny, lbm_storage storage, lbm_bc bc, int host_io) {
    if (nx < 1 || ny < 1 || storage < LBM_F64 || storage > LBM_BF16DEV || bc < LBM_BC_DIRICHLET_EQ ||
        bc > LBM_BC_CHANNEL || (host_io != 0 && host_io != 1))
        return 0;
    // the allocations of lbm_create, setup_tma and ensure_staging, in that order
    const size_t es = lbm::storage_bytes(storage);
    const size_t per_row = (static_cast<size_t>(nx) * es + 127) / 128 * 128 / es;
    const size_t cts = storage == LBM_F64 ? 8 : 4;
    size_t bytes = 2 * 9 * per_row * static_cast<size_t>(ny) * es;
    bytes += static_cast<size_t>(nx + ny) * 4 * cts;
    bytes += sizeof(double) * (lbm::kDiagBlocks * lbm::kDiag + lbm::kDiag) + 256;
    if (bc == LBM_BC_CHANNEL) bytes += kGraphChunk * (sizeof(double) + 9 * sizeof(float));
    if (storage == LBM_F32 && bc == LBM_BC_DIRICHLET_EQ) bytes += 256;
    if (host_io) bytes += 3 * sizeof(double) * static_cast<size_t>(nx) * ny;
    return bytes;
}

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int lbm_create(int nx, int ny, lbm_storage storage, double rho0, double ux0, double uy0,
               const lbm_rates* rates, lbm_bc bc, void* cuda_stream, const lbm_allocator* alloc,
               lbm_handle* out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || (long long)nx * ny > 2147483647LL)
        return fail(nullptr, LBM_ERR_ARG, "lattice size out of range");
    if (storage < LBM_F64 || storage > LBM_BF16DEV) return fail(nullptr, LBM_ERR_ARG, "bad storage");
    if (bc != LBM_BC_DIRICHLET_EQ && bc != LBM_BC_PERIODIC && bc != LBM_BC_CHANNEL)
        return fail(nullptr, LBM_ERR_ARG, "bad bc");
    if (bc == LBM_BC_CHANNEL && nx < 2) return fail(nullptr, LBM_ERR_ARG, "the channel needs nx >= 2");
    if (!rates) return fail(nullptr, LBM_ERR_ARG, "rates is NULL");
    if (!(rho0 > 0) || !is_finite(rho0) || !is_finite(ux0) || !is_finite(uy0))
        return fail(nullptr, LBM_ERR_ARG, "far-field state must be finite with rho0 > 0");
    int warn = LBM_OK;
    for (int i = 0; i < 9; ++i) {
        if (!is_finite(rates->s[i])) return fail(nullptr, LBM_ERR_ARG, "non-finite relaxation rate");
        if (!(rates->s[i] > 0 && rates->s[i] < 2)) warn = LBM_WARN_UNSTABLE_PARAMS;
    }
    if (!is_finite(rates->n) || !is_finite(rates->m) || rates->n < 0 || rates->m < 0)
        return fail(nullptr, LBM_ERR_ARG, "Guo weights n, m must be finite and >= 0");
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(nullptr, LBM_ERR_ARG, "allocator lacks alloc or free");

    lbm_ctx* h = new lbm_ctx();
    h->nx = nx;
    h->ny = ny;
    h->storage = storage;
    h->bc = bc;
    h->rho0 = rho0;
    h->ux0 = ux0;
    h->uy0 = uy0;
    h->rates = *rates;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    if (alloc) {
        h->alloc = *alloc;
        h->custom_alloc = true;
    }
    h->rho_f = rho0;
    h->ux_f = ux0;
    h->uy_f = uy0;
    h->bulk[0] = 0;  // no layer until lbm_set_sponge
    h->bulk[1] = nx;
    h->bulk[2] = 0;
    h->bulk[3] = ny;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    const size_t es = lbm::storage_bytes(storage);
    const long long per_row = (long long)((nx * es + 127) / 128 * 128 / es);
    h->geo = Geometry{nx, ny, per_row, per_row * ny};
    h->buf_bytes = 9 * (size_t)h->geo.plane * es;
    const size_t cts = storage == LBM_F64 ? 8 : 4;
    if (h->geo.plane > 2147483647LL) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "lattice too large: one plane must hold fewer than 2^31 elements");
    }
    h->chi_bytes_x = (size_t)nx * 4 * cts;
    h->chi_bytes_y = (size_t)ny * 4 * cts;
    h->diag_bytes = sizeof(double) * (lbm::kDiagBlocks * lbm::kDiag + lbm::kDiag);
    h->buf[0] = dev_alloc(h, h->buf_bytes);
    h->buf[1] = dev_alloc(h, h->buf_bytes);
    h->chi_x = dev_alloc(h, h->chi_bytes_x);
    h->chi_y = dev_alloc(h, h->chi_bytes_y);
    h->diag = static_cast<double*>(dev_alloc(h, h->diag_bytes));
    h->d_time = static_cast<long long*>(dev_alloc(h, 256));
    if (bc == LBM_BC_CHANNEL)
        h->d_src_table = static_cast<double*>(
            dev_alloc(h, kGraphChunk * (sizeof(double) + 9 * sizeof(float))));
    if (!h->buf[0] || !h->buf[1] || !h->chi_x || !h->chi_y || !h->diag || !h->d_time ||
        (bc == LBM_BC_CHANNEL && !h->d_src_table)) {
        lbm_destroy(h);
        return fail(nullptr, LBM_ERR_OOM, "device allocation failed");
    }
    // zero the absorbing strength and both buffers (a zero deviation is the far-field state)
    e = cudaMemsetAsync(h->chi_x, 0, h->chi_bytes_x, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->chi_y, 0, h->chi_bytes_y, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[0], 0, h->buf_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, h->buf_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_time, 0, sizeof(long long), h->stream);
    for (int i = 0; i < 2 && e == cudaSuccess && lbm::canary_requested(); ++i)
        e = lbm::paint_canary(h->buf[i], es, nx, h->geo.pitch, 9ll * ny, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        lbm_destroy(h);
        return cuda_fail(nullptr, e, "initial clear");
    }
    refresh_consts(h);
    h->cpt = pair_kernel_ok(h) ? 2 : 1;
    if (const char* c = std::getenv("LBM_CPT")) {
        if (!std::strcmp(c, "1")) h->cpt = 1;
    }
    // Two steps per launch pay off once the double-buffered state no longer
    // fits in L2 (the step is then HBM-bound); below that the extra ring of
    // collisions costs more than the traffic it saves.
    int l2 = 0;
    if (h->cpt == 2 && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) == cudaSuccess &&
        2 * h->buf_bytes > static_cast<size_t>(l2))
        h->spl = 2;
    if (const char* c = std::getenv("LBM_SPL")) {
        if (!std::strcmp(c, "2") && h->cpt == 2) h->spl = 2;
        if (!std::strcmp(c, "1")) h->spl = 1;
    }
    if (bc == LBM_BC_CHANNEL) h->spl = 1;  // the two-step tiles have no channel edges
    // FP32 Dirichlet lattices whose state exceeds four times L2 stage the
    // two-step tiles' input by TMA: measured 2-8 % ahead of plain loads from
    // 4096^2 up, 3 % behind at 2048^2 (LBM_TMA=0 or 1 overrides the choice).
    // 16-bit storage can be staged too (LBM_TMA=1), measured level with plain loads.
    const char* tma_env = std::getenv("LBM_TMA");
    bool want_tma = storage == LBM_F32 && h->spl == 2 &&
                    2 * h->buf_bytes > 4 * static_cast<size_t>(l2);
    if (tma_env) want_tma = std::strcmp(tma_env, "0") != 0;
    if (storage != LBM_F64 && bc == LBM_BC_DIRICHLET_EQ && want_tma)
        h->tma = setup_tma(h) == LBM_OK;
    h->err.clear();
    set_source_shape(h);
    if (const char* m = std::getenv("LBM_LAUNCH")) {
        if (!std::strcmp(m, "plain")) h->launch_mode = kLaunchPlain;
        else if (!std::strcmp(m, "pdl")) h->launch_mode = kLaunchPdl;
        else if (!std::strcmp(m, "graph")) h->launch_mode = kLaunchGraph;
    }
    *out = h;
    if (warn) g_create_error = "a relaxation rate lies outside (0, 2)";
    return warn;
}

int lbm_set_sponge(lbm_handle h, lbm_variant variant, const double* chi_x, const double* chi_y,
                   double rho_ref, double ux_ref, double uy_ref) {
    if (!h) return LBM_ERR_ARG;
    if (variant < LBM_SPONGE_NONE || variant > LBM_SPONGE_VISCOUS) return fail(h, LBM_ERR_ARG, "bad variant");
    if (variant == LBM_SPONGE_VISCOUS && chi_x && chi_y) {
        for (int i = 0; i < h->nx; ++i)
            if (chi_x[i] > 1.0) return fail(h, LBM_ERR_ARG, "viscous sponge: layer fraction above 1");
        for (int i = 0; i < h->ny; ++i)
            if (chi_y[i] > 1.0) return fail(h, LBM_ERR_ARG, "viscous sponge: layer fraction above 1");
    }
    if (!chi_x || !chi_y) return fail(h, LBM_ERR_ARG, "chi arrays are NULL");
    if (!(rho_ref > 0) || !is_finite(rho_ref) || !is_finite(ux_ref) || !is_finite(uy_ref))
        return fail(h, LBM_ERR_ARG, "reference state must be finite with rho_ref > 0");
    double chi_max = 0.0;
    for (int i = 0; i < h->nx; ++i) {
        if (!(chi_x[i] >= 0) || !is_finite(chi_x[i])) return fail(h, LBM_ERR_ARG, "chi_x must be finite and >= 0");
        chi_max = std::fmax(chi_max, chi_x[i]);
    }
    for (int i = 0; i < h->ny; ++i) {
        if (!(chi_y[i] >= 0) || !is_finite(chi_y[i])) return fail(h, LBM_ERR_ARG, "chi_y must be finite and >= 0");
        chi_max = std::fmax(chi_max, chi_y[i]);
    }
    DeviceGuard dg(h->device);
    cudaError_t e;
    // Per-axis tables {chi, 1/(1 + n chi), 1/(1 + m chi), 0}, the factors in FP64.
    const double nn = h->rates.n, mm = h->rates.m;
    if (h->storage == LBM_F64) {
        std::vector<double> tx(4 * (size_t)h->nx), ty(4 * (size_t)h->ny);
        for (int i = 0; i < h->nx; ++i) {
            tx[4 * i] = chi_x[i]; tx[4 * i + 1] = 1.0 / (1.0 + nn * chi_x[i]);
            tx[4 * i + 2] = 1.0 / (1.0 + mm * chi_x[i]); tx[4 * i + 3] = 0.0;
        }
        for (int i = 0; i < h->ny; ++i) {
            ty[4 * i] = chi_y[i]; ty[4 * i + 1] = 1.0 / (1.0 + nn * chi_y[i]);
            ty[4 * i + 2] = 1.0 / (1.0 + mm * chi_y[i]); ty[4 * i + 3] = 0.0;
        }
        e = cudaMemcpyAsync(h->chi_x, tx.data(), h->chi_bytes_x, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->chi_y, ty.data(), h->chi_bytes_y, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    } else {
        std::vector<float> tx(4 * (size_t)h->nx), ty(4 * (size_t)h->ny);
        for (int i = 0; i < h->nx; ++i) {
            tx[4 * i] = (float)chi_x[i]; tx[4 * i + 1] = (float)(1.0 / (1.0 + nn * chi_x[i]));
            tx[4 * i + 2] = (float)(1.0 / (1.0 + mm * chi_x[i])); tx[4 * i + 3] = 0.0f;
        }
        for (int i = 0; i < h->ny; ++i) {
            ty[4 * i] = (float)chi_y[i]; ty[4 * i + 1] = (float)(1.0 / (1.0 + nn * chi_y[i]));
            ty[4 * i + 2] = (float)(1.0 / (1.0 + mm * chi_y[i])); ty[4 * i + 3] = 0.0f;
        }
        e = cudaMemcpyAsync(h->chi_x, tx.data(), h->chi_bytes_x, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->chi_y, ty.data(), h->chi_bytes_y, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_sponge copy");
    drop_graphs(h);  // the captured launches carry the old constants
    h->variant = variant;
    h->rho_f = rho_ref;
    h->ux_f = ux_ref;
    h->uy_f = uy_ref;
    lbm::zero_run(chi_x, h->nx, h->bulk[0], h->bulk[1]);
    lbm::zero_run(chi_y, h->ny, h->bulk[2], h->bulk[3]);
    refresh_consts(h);
    const double s_nu = h->rates.s[7];
    if ((variant == LBM_SPONGE_II || variant == LBM_SPONGE_III) && chi_max > 4.0 / s_nu)
        return fail(h, LBM_WARN_UNSTABLE_PARAMS, "max chi exceeds the critical value 4/s");
    if (variant == LBM_SPONGE_I && s_nu + chi_max > 2.0)
        return fail(h, LBM_WARN_UNSTABLE_PARAMS, "type I with s + chi > 2 is unstable");
    return LBM_OK;
}

int lbm_init_equilibrium(lbm_handle h, const double* rho, const double* ux, const double* uy,
                         int on_device) {
    if (!h) return LBM_ERR_ARG;
    if (!rho || !ux || !uy) return fail(h, LBM_ERR_ARG, "field pointer is NULL");
    DeviceGuard dg(h->device);
    const double *dr = rho, *dx = ux, *dy = uy;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        int rc = ensure_staging(h);
        if (rc) return rc;
        const size_t n = (size_t)h->nx * h->ny;
        double* s = h->staging;
        e = cudaMemcpyAsync(s, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s + n, ux, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s + 2 * n, uy, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "lbm_init_equilibrium upload");
        dr = s;
        dx = s + n;
        dy = s + 2 * n;
    }
    h->cur = 0;
    e = lbm::launch_init(h->storage, h->buf[0], h->geo, base_of(h), dr, dx, dy, h->bc, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_init_equilibrium");
    h->initialised = true;
    h->time = 0;
    e = cudaMemsetAsync(h->d_time, 0, sizeof(long long), h->stream);  // the line source's clock
    if (e != cudaSuccess) return cuda_fail(h, e, "clock reset");
    return LBM_OK;
}

int lbm_init_pulse(lbm_handle h, double eps, double half_width, double x0, double y0) {
    if (!h) return LBM_ERR_ARG;
    if (!is_finite(eps) || !(half_width > 0) || !is_finite(half_width) || !is_finite(x0) ||
        !is_finite(y0))
        return fail(h, LBM_ERR_ARG, "pulse parameters must be finite with half_width > 0");
    DeviceGuard dg(h->device);
    h->cur = 0;
    cudaError_t e = lbm::launch_init_pulse(h->storage, h->buf[0], h->geo, base_of(h), eps,
                                           half_width, x0, y0, h->bc, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_init_pulse");
    h->initialised = true;
    h->time = 0;
    e = cudaMemsetAsync(h->d_time, 0, sizeof(long long), h->stream);  // the line source's clock
    if (e != cudaSuccess) return cuda_fail(h, e, "clock reset");
    return LBM_OK;
}

int lbm_step(lbm_handle h, int nsteps) {
    const lbm::NvtxRange nvtx("lbm_step");
    if (!h) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lbm_step before lbm_init_equilibrium / lbm_set_state");
    DeviceGuard dg(h->device);
    cudaError_t e = cudaSuccess;
    const bool pdl = h->launch_mode != kLaunchPlain;
    if (h->launch_mode == kLaunchGraph && nsteps >= kGraphChunk) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(h->stream, &cs);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamIsCapturing");
        if (cs == cudaStreamCaptureStatusNone) {
            e = ensure_graph(h, h->cur);
            if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step graph build");
            while (nsteps >= kGraphChunk) {
                e = cudaGraphLaunch(h->graph[h->cur], h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step graph launch");
                h->time += kGraphChunk;  // an even number of launches leaves cur unchanged
                nsteps -= kGraphChunk;
            }
        }
    }
    // the channel issues at most kGraphChunk launches per source table
    while (nsteps > 0) {
        const bool channel = h->bc == LBM_BC_CHANNEL;
        const int chunk = channel && nsteps > kGraphChunk ? kGraphChunk : nsteps;
        if (channel) {
            e = launch_source_table(h, h->stream, chunk);
            if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step source table");
        }
        int issued = 0;
        while (issued < chunk) {
            const int n = (h->spl == 2 && chunk - issued >= 2) ? 2 : 1;
            e = n == 2 ? launch_two_steps(h, h->buf[h->cur], h->buf[1 - h->cur], h->stream, pdl)
                       : launch_one_step(h, h->buf[h->cur], h->buf[1 - h->cur], h->stream, pdl,
                                         issued);
            if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step launch");
            h->cur = 1 - h->cur;
            h->time += n;
            issued += n;
        }
        nsteps -= chunk;
        if (channel) {  // the line source's clock
            advance_time_kernel<<<1, 1, 0, h->stream>>>(h->d_time, issued);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step clock");
        }
    }
    return LBM_OK;
}

int lbm_moments(lbm_handle h, double* rho_dev, double* ux, double* uy, int on_device) {
    if (!h) return LBM_ERR_ARG;
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lbm_moments before initialisation");
    DeviceGuard dg(h->device);
    const size_t n = (size_t)h->nx * h->ny;
    double *dr = rho_dev, *dx = ux, *dy = uy;
    if (!on_device) {
        int rc = ensure_staging(h);
        if (rc) return rc;
        dr = rho_dev ? h->staging : nullptr;
        dx = ux ? h->staging + n : nullptr;
        dy = uy ? h->staging + 2 * n : nullptr;
    }
    cudaError_t e = lbm::launch_moments(h->storage, h->buf[h->cur], h->geo, base_of(h), h->bc, dr, dx,
                                        dy, h->stream, readout_source(h));
    if (e == cudaSuccess && !on_device) {
        if (rho_dev) e = cudaMemcpyAsync(rho_dev, dr, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && ux) e = cudaMemcpyAsync(ux, dx, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && uy) e = cudaMemcpyAsync(uy, dy, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_moments");
    return on_device ? LBM_OK : check_tma(h);
}

int lbm_diagnostics(lbm_handle h, int x0, int y0, int x1, int y1, double out[6]) {
    if (!h) return LBM_ERR_ARG;
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lbm_diagnostics before initialisation");
    if (x0 < 0 || y0 < 0 || x1 > h->nx || y1 > h->ny || x0 > x1 || y0 > y1)
        return fail(h, LBM_ERR_ARG, "region outside the lattice");
    DeviceGuard dg(h->device);
    double* partial = h->diag;
    double* res = h->diag + lbm::kDiagBlocks * lbm::kDiag;
    cudaError_t e = lbm::launch_diagnostics(h->storage, h->buf[h->cur], h->geo, base_of(h), h->bc, x0, y0,
                                            x1, y1, partial, res, h->stream, readout_source(h));
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, lbm::kDiag * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_diagnostics");
    if (const int rc = check_tma(h)) return rc;
    if (out[5] > 0) return fail(h, LBM_ERR_NONFINITE, "the state holds non-finite values");
    return LBM_OK;
}

size_t lbm_state_bytes(lbm_handle h) { return h ? h->buf_bytes : 0; }

int lbm_get_state(lbm_handle h, void* dst, size_t bytes, int on_device, int64_t* time) {
    if (!h) return LBM_ERR_ARG;
    if (!dst || bytes != h->buf_bytes) return fail(h, LBM_ERR_ARG, "dst / bytes do not match lbm_state_bytes");
    DeviceGuard dg(h->device);
    cudaError_t e = cudaMemcpyAsync(dst, h->buf[h->cur], bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_get_state");
    if (time) *time = h->time;
    return on_device ? LBM_OK : check_tma(h);
}

int lbm_set_state(lbm_handle h, const void* src, size_t bytes, int on_device, int64_t time) {
    if (!h) return LBM_ERR_ARG;
    if (!src || bytes != h->buf_bytes) return fail(h, LBM_ERR_ARG, "src / bytes do not match lbm_state_bytes");
    if (time < 0) return fail(h, LBM_ERR_ARG, "time < 0");
    DeviceGuard dg(h->device);
    h->cur = 0;
    cudaError_t e = cudaMemcpyAsync(h->buf[0], src, bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_state");
    h->time = time;
    h->initialised = true;
    e = cudaMemcpyAsync(h->d_time, &h->time, sizeof(long long), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "clock set");
    return LBM_OK;
}

int64_t lbm_time(lbm_handle h) { return h ? h->time : -1; }

int lbm_set_launch_mode(lbm_handle h, int mode) {
    if (!h) return LBM_ERR_ARG;
    if (mode < kLaunchPlain || mode > kLaunchGraph) return fail(h, LBM_ERR_ARG, "bad launch mode");
    h->launch_mode = mode;
    return LBM_OK;
}

int lbm_set_cells_per_thread(lbm_handle h, int cells) {
    if (!h) return LBM_ERR_ARG;
    if (cells != 1 && cells != 2) return fail(h, LBM_ERR_ARG, "cells per thread must be 1 or 2");
    if (cells == 2 && !pair_kernel_ok(h))
        return fail(h, LBM_ERR_ARG, "two cells per thread needs FP32 or 16-bit storage and 9 planes below 2^32 elements");
    if (cells == 2 && h->arith == LBM_ARITH_COMPENSATED)
        return fail(h, LBM_ERR_ARG, "compensated arithmetic steps one cell per thread");
    if (cells != h->cpt) {
        DeviceGuard dg(h->device);
        cudaStreamSynchronize(h->stream);
        drop_graphs(h);  // the captured launches name the other kernel
        h->cpt = cells;
        if (cells == 1) h->spl = 1;
    }
    return LBM_OK;
}

int lbm_set_steps_per_launch(lbm_handle h, int steps) {
    if (!h) return LBM_ERR_ARG;
    if (steps != 1 && steps != 2) return fail(h, LBM_ERR_ARG, "steps per launch must be 1 or 2");
    if (steps == 2 && h->cpt != 2)
        return fail(h, LBM_ERR_ARG, "two steps per launch needs two cells per thread");
    if (steps == 2 && h->bc == LBM_BC_CHANNEL)
        return fail(h, LBM_ERR_ARG, "two steps per launch is not available for the channel boundary");
    if (steps != h->spl) {
        DeviceGuard dg(h->device);
        cudaStreamSynchronize(h->stream);
        drop_graphs(h);  // the captured launches name the other kernel
        h->spl = steps;
    }
    return LBM_OK;
}

int lbm_steps_per_launch(lbm_handle h) { return h ? h->spl : LBM_ERR_ARG; }

int lbm_set_arithmetic(lbm_handle h, lbm_arithmetic a) {
    if (!h) return LBM_ERR_ARG;
    if (a != LBM_ARITH_NATIVE && a != LBM_ARITH_COMPENSATED)
        return fail(h, LBM_ERR_ARG, "arithmetic must be LBM_ARITH_NATIVE or LBM_ARITH_COMPENSATED");
    if (a == LBM_ARITH_COMPENSATED && h->storage != LBM_F32)
        return fail(h, LBM_ERR_ARG, "compensated arithmetic needs LBM_F32 storage");
    if (a == h->arith) return LBM_OK;
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);  // the captured launches name the other kernel
    h->arith = a;
    if (a == LBM_ARITH_COMPENSATED) {  // one cell, one step per launch
        h->cpt = 1;
        h->spl = 1;
        h->tma = false;
    }
    return LBM_OK;
}

int lbm_get_arithmetic(lbm_handle h) { return h ? h->arith : LBM_ERR_ARG; }

int lbm_set_tma_staging(lbm_handle h, int on) {
    if (!h) return LBM_ERR_ARG;
    if (on != 0 && on != 1) return fail(h, LBM_ERR_ARG, "on must be 0 or 1");
    if (on == (h->tma ? 1 : 0)) return LBM_OK;
    if (on && h->arith == LBM_ARITH_COMPENSATED)
        return fail(h, LBM_ERR_ARG, "compensated arithmetic steps one cell, one step per launch");
    DeviceGuard dg(h->device);
    if (on) {
        const int rc = setup_tma(h);
        if (rc != LBM_OK) return rc;
    }
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);  // the captured launches name the other kernel
    h->tma = on == 1;
    return LBM_OK;
}

int lbm_tma_staging(lbm_handle h) { return h ? (h->tma ? 1 : 0) : LBM_ERR_ARG; }

int lbm_set_source(lbm_handle h, double amplitude, double omega, double phase) {
    if (!h) return LBM_ERR_ARG;
    if (h->bc != LBM_BC_CHANNEL) return fail(h, LBM_ERR_ARG, "a line source needs the channel boundary");
    if (!std::isfinite(amplitude) || !std::isfinite(omega) || !std::isfinite(phase))
        return fail(h, LBM_ERR_ARG, "source parameters must be finite");
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);  // the captured launches carry the old source
    h->src.amp = amplitude;
    h->src.omega = omega;
    h->src.phase = phase;
    return LBM_OK;
}

int lbm_cells_per_thread(lbm_handle h) { return h ? h->cpt : LBM_ERR_ARG; }

int lbm_set_stream(lbm_handle h, void* cuda_stream) {
    if (!h) return LBM_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return LBM_OK;
}

void lbm_destroy(lbm_handle h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    dev_free(h, h->buf[0], h->buf_bytes);
    dev_free(h, h->buf[1], h->buf_bytes);
    dev_free(h, h->chi_x, h->chi_bytes_x);
    dev_free(h, h->chi_y, h->chi_bytes_y);
    dev_free(h, h->diag, h->diag_bytes);
    dev_free(h, h->d_time, 256);
    dev_free(h, h->d_src_table, kGraphChunk * (sizeof(double) + 9 * sizeof(float)));
    dev_free(h, h->tma_err, 256);
    dev_free(h, h->staging, h->staging_bytes);
    delete h;
}

}  // extern "C"
