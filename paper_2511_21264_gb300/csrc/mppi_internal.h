// Internal (non-ABI) declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <vector>

namespace mppi {

// NVTX range for the lifetime of a scope (shows up in nsys / ncu timelines;
// costs nothing when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// bits of a controller's device error word
constexpr int ERRB_NONFINITE = 1;
constexpr int ERRB_CHOLESKY = 2;
constexpr int ERRB_TIMEOUT = 4;

struct DevModel;
struct DevTask;

struct HostModelInfo {
    int na = 0, nb = 0;
    std::vector<float> x0;
};

// Arguments of the rollout kernel (one group of lanes per sample).
struct RolloutArgs {
    const DevModel* model;
    int n;                       // samples
    int H;                       // horizon
    const float* states;         // n x nx (stride state_stride; 0 = one shared state)
    int state_stride;
    const float* U;              // explicit controls n x H x nu (MODE 0)
    const float* u_nom;          // H x nu (MODE 1)
    const float* sigma;          // nu (MODE 1)
    uint64_t seed;               // Philox key (MODE 1)
    const unsigned long long* iter_ptr;  // iteration counter on the device, or null
    unsigned long long iter_val;         // iteration when iter_ptr is null
    float* costs;                // n
    float* states_out;           // optional n x nx
    int* err;                    // error word
    int stage_unom;              // stage u_nom in shared memory
    unsigned long long* stats;   // optional: [sample-steps, contacts, exact box tests]
    float* U_store;              // optional: sampled controls, H x n x nu (h-major), MODE 1
    int U_hmajor;                // MODE 0: U is H x n x nu (h-major) instead of n x H x nu
    const float* Lfac;           // optional: covariance factors H x nu x nu (MODE 1), else diagonal sigma
    const DevTask* task;         // optional: the ball-task cost suite replaces the stage cost
    int pdl;                     // launch as a programmatic dependent of the previous kernel
    int lps;                     // lanes per sample: 32, 16 or 8 (0 = 32)
    int place;                   // lone ball contact solve: 0 fused with the arms' factor, 1 after it
};

// Arguments of the weighted-mean update (one CTA per horizon step).
struct UpdateArgs {
    int K;
    int H;              // horizon (rows of u_nom / u_out); set by the launch
    const float* costs;
    const float* u_nom;
    float* u_out;
    const float* sigma;
    const float* u_lo;
    const float* u_hi;
    float lambda;
    uint64_t seed;
    unsigned long long* iter_ptr;
    unsigned long long iter_val;
    int* err;
    float* best;        // optional: min cost, argmin
    int advance;        // last CTA increments *iter_ptr
    unsigned int* done; // CTA completion counter (reset by the last CTA)
    const float* U_stored;  // optional: the rollout's sampled controls (H x K x nu), else regenerated
    int pdl;                // launch as a programmatic dependent of the previous kernel
};

struct NoiseArgs {
    int K, H;
    const float* sigma;
    uint64_t seed;
    uint64_t iter;
    float* eps;
};

// accessors of the opaque model handle for the other translation units
}  // namespace mppi
struct mppi_model;
namespace mppi {
const DevModel* model_device(const mppi_model* m);
void model_bounds(const mppi_model* m, int j, float* lo, float* hi);
float model_dt(const mppi_model* m);

// descriptor of one controller in a batched iteration (device table)
struct BatchInst {
    const DevModel* model;
    const float* state;
    float* u;  // nominal controls, updated in place
    float* costs;
    const float* sigma;
    const float* u_lo;
    const float* u_hi;
    unsigned long long* iter;
    unsigned int* done;
    int* err;
    float* best;
    unsigned long long seed;
    int K, H;
    float lambda;
    int stage_unom;
    int tile0;  // first work item (tile of samples) of this instance
    int row0;   // first update CTA of this instance
    // the full Eq. 8 update (elite != 0: elite set, learning rate,
    // covariance blocks) and the projected samples (Eq. 5)
    int elite, n_elite, update_cov, cov_sampling;
    float eta, cov_floor;
    float* Sigma;               // H x nu x nu
    float* Lfac;                // H x nu x nu sampling factors (rewritten by the covariance update)
    unsigned long long* sel;    // [threshold key, best key, finite count]
    int* eidx;                  // K elite indices
    float* U;                   // H x K x nu projected samples, or null (samples drawn in the rollout)
};

struct BatchCtl {
    unsigned int next;    // next tile to take
    unsigned int exited;  // CTAs that finished
};

// launch shape of the persistent batched rollout
struct BatchLaunch {
    int na = 7, spc = 4, lps = 32, place = 0, grid = 0, max_unom = 0;
    size_t smem = 0;
    int mode = 1;       // 1: samples drawn in the rollout; 0: every instance's projected samples (BatchInst::U)
    int sel_P = 0;      // > 0: some instance uses the elite set; its sort holds up to sel_P keys
};
// spc: samples per tile (rounded up to whole warps); lps: lanes per sample
// (32, 16 or 8; 0 = 32); place: the lone ball contact's solve fused (0) or
// after the arms' factor (1)
int batch_shape(int na, int spc, int lps, int place, int max_h, BatchLaunch* L);
int launch_batch_iteration(const BatchInst* insts, int n, int ntiles, int nrows, BatchCtl* ctl, const BatchLaunch& L,
                           cudaStream_t s);
int launch_shift(float* u, int H, int nu, cudaStream_t s);

// QP smoothing projection (Eq. 5): one class of sequences (a joint)
struct QPClass {
    float lo[4], hi[4];  // bounds on position, velocity, acceleration, jerk
    float s[4];          // row-group scales; 0 marks a free group (both bounds infinite)
    float rho;           // ADMM penalty
    float pad[3];
};

// Arguments of the projection kernel (one thread per sequence).  Sequence i
// belongs to class i / per_cls as member i % per_cls; element h of its input
// and output sits at (member * a + class * b + h * h_stride).
struct QPArgs {
    int n, H, iters, per_cls;
    float dt;
    const QPClass* cls;  // classes
    const float4* band;  // per class 2H: forward then backward band factor rows
    const float* q0;     // present position, per sequence (q_per_seq) or per class
    const float* qd0;    // present velocity, same indexing
    int q_per_seq;
    const float* vin;    // explicit input, or null to sample (member = sample k, class = joint j)
    long long i_a, i_b, i_h;
    // sampling: v = u_nom[h, j] + sigma_j z_j, or + (L_h z)_j with Lfac (no clamp)
    int nu;
    const float* u_nom;
    const float* sigma;
    const float* Lfac;
    uint64_t seed;
    const unsigned long long* iter_ptr;
    unsigned long long iter_val;
    float* out;
    long long o_a, o_b, o_h;
    const float* minv;   // H <= 32: per class the 32 x 32 inverse (I + rho D^T D)^-1 in velocity coordinates
    // extents, for the bounds-check build: classes, floats of vin and of out
    int n_cls;
    long long in_n, out_n;
};
constexpr int QP_WARP_MAX_H = 32;
int qp_band_factor(int H, double rho, const double sc[4], float4* band);
int qp_dense_inverse(int H, double rho, const double sc[4], float* minv);
void qp_make_class(const float b[8], const float sc[4], float rho, QPClass* c);
int qp_validate(const float b[8], const float sc[4], float rho);
int launch_qp(const QPArgs& a, cudaStream_t s);
int qp_build(int nu, int H, const float* bounds, float rho, const float* scales, std::vector<unsigned char>& host);
QPArgs qp_controller_args(int nu, int nq, int K, int H, int iters, float dt, const void* d_qp, const float* state,
                          const float* u_nom, const float* sigma, const float* Lfac, uint64_t seed,
                          const unsigned long long* iter_ptr, float* U);

// closed-loop episode helpers
int launch_best_average(const float* U, const float* best, const float* bestU, int K, int nu, int n, float* u1,
                        cudaStream_t s);
int launch_shift_rows(float* u, int H, int row, int n, cudaStream_t s);
int launch_probe(int na, const DevModel* model, const float* x, float* out, cudaStream_t s);

// bounds words of the translation units with kernels (read and cleared;
// always 0 unless built with -DMPPI_BOUNDS_CHECK)
unsigned bounds_word_api();
unsigned bounds_word_batch();
unsigned bounds_word_qp();
unsigned bounds_word_loop();
unsigned bounds_word_rollout7();
unsigned bounds_word_rollout3();

int parse_model_blob(const void* blob, size_t len, DevModel* out, HostModelInfo* info);
int launch_rollout(int na, int mode, const RolloutArgs& a, int spc, cudaStream_t s);
int launch_update(int nu, const UpdateArgs& a, int H, cudaStream_t s);
int launch_noise(int nu, const NoiseArgs& a, cudaStream_t s);

}  // namespace mppi
