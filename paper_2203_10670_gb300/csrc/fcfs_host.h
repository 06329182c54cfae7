// Host-side helpers shared by the libfcfs translation units.
#pragma once

#include <stdarg.h>

#include <nvtx3/nvToolsExt.h>

#include "fcfs_internal.cuh"

namespace fcfs {

// A named NVTX range for the duration of a scope: the C-ABI calls and the
// serving loop's steps appear by name on profiler timelines (no cost without
// an attached tool beyond a few instructions).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct TileChoice {
    int WX, WY, WD;  // windows per tile along x, y, depth
    int G = 0;       // thread groups per output column (0: planner default)
    int tma = -1;    // 1: TMA-staged persistent kernel, 0: gather kernel, -1: best available
    int threads = 0; // CTA size of the TMA-staged kernel (0: 256)
    int rs = 1;      // 1: register-blocked variant when one is compiled for (r, span), 0: per-output kernel
    int psk = 0;     // 1: polyphase strip kernel when the descriptor is in its scope (2D), 0: tile kernels
};

int fail(int status, const char* fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char* what);

double kernel_value(int method, double t, double ka);
double keys_a(const fcfs_desc* d);
int support_radius(int method);
int k_min(int method, int s);
long long out_len(long long n, int r, int s);
int template_taps(int nt);
int axis_taps(const fcfs_desc* d, int a);
int fixed_taps(int method, int r, int s, int align, double ka, int aa);

int validate_axis(const fcfs_axis& a, int idx);
int validate_desc(const fcfs_desc* d, bool output_dtype_check);
long long numel_in(const fcfs_desc* d);
long long numel_out(const fcfs_desc* d);
int dtype_size(int dt);

void fill_axis(AxisP* A, const fcfs_axis& a, long long n_in, int C, int nt_kernel, int align, double ka, int aa);
void identity_axis(AxisP* A, int nt_kernel);

int build_forward_params(const fcfs_desc* d, const void* x, void* y, FwdParams* out, int* ntk);
void apply_tiles(FwdParams& P, bool is3d, int WX, int WY, int WD, int G = 0);
bool tma_eligible(const fcfs_desc* d, const void* x);
int prepare_tma(const fcfs_desc* d, const FwdParams& P, TmaFwdParams* T, int threads = 256);
TileChoice default_tma_tiles(const FwdParams& P, int es, bool is3d = false);
int prepare_tma3(const fcfs_desc* d, const FwdParams& P, TmaFwd3Params* T, int threads = 256);
size_t forward3_tma_smem_bytes(const TmaFwd3Params& T);
int launch_choice(const fcfs_desc* d, FwdParams& P, int ntk, const TileChoice& t, cudaStream_t st);
TileChoice default_tiles(const FwdParams& P, bool is3d);
void set_plan(const FwdParams& P, int ndim, int din, int dout, TileChoice t);
void clear_plans();
int plan_count();
bool get_plan(const FwdParams& P, int ndim, int din, int dout, TileChoice* t);
int launch_planned(FwdParams& P, int ntk, bool is3d, int din, int dout, cudaStream_t st);
int forward_planned(const fcfs_desc* d, const void* x, void* y, const Epi* epi, cudaStream_t st);
bool forward_has_epilogue_path(const fcfs_desc* d, const void* x);
int fused_forward_tc(const fcfs_desc* d, const fcfs_epilogue* e, const void* x, void* y, cudaStream_t st);
int read_status_fused_tc(int clear);
int build_adjoint(const AxisP& A, AdjAxis* J);
int build_adjp(const AxisP& A, AdjP* J);
void plan_dx(BwdParams& B, bool is3d);
void plan_dx_region(BwdParams& B, int x0, int x1, int y0, int y1);

// polyphase strip kernels (fcfs_psk_host.cu): FCFS_OK when launched, -1 when the
// descriptor is outside their scope (the caller takes another kernel), else an error
int psk_forward(const fcfs_desc* d, const FwdParams& F, cudaStream_t st);
int psk_input_gradient(const fcfs_desc* d, const BwdParams& B, const void* gy, void* gx, int ntk, cudaStream_t st);
bool psk_enabled();
int psk_policy();  // 0 never, 1 default, 2 wherever in scope

// non-separable 2D kernels (fcfs_full2d.cu)
int full2d_forward(const fcfs_desc* d, const void* x, void* y, cudaStream_t st);
size_t full2d_workspace(const fcfs_desc* d);
int full2d_backward(const fcfs_desc* d, const void* x, const void* gy, void* gx, float* gw, void* ws,
                    size_t ws_bytes, cudaStream_t st);

}  // namespace fcfs
