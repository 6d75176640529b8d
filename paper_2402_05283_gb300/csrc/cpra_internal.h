// cpra_internal.h - plan layout and kernel launchers shared by the .cu files.
//
// Device data of one plan (all stacks contiguous per angle):
//   g, g_alt   [Np][N][N]    float   iterate (Jacobi double buffer for Eq. 4)
//   Hp         [Np][N][N/2]  float2  row spectra of g, packed: column 0 holds
//                                    (Re H(y,0), Re H(y,N/2)); the two-pass
//                                    engine keeps it between its passes
//   A_main     [Np][N/2][N]  float   Hermitian-symmetrised amplitude, kx < N/2,
//                                    column-major ([kx][ky])
//   A_nyq      [Np][N]       float   the same at kx = N/2
//   Cn, sumA2  [Np]          double  antisymmetric-part energy, sum A^2
//   S          [Np][N][W]    uint32  support bits, W = ceil(N/32) words a row
//   err_acc    [Np]          double  per-iteration error accumulator
//   err_hist   [cap][Np]     double  Fourier error history
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "cpra.h"

namespace cpra {

struct JobStatic;
struct JobStep;

// Device-side status of a plan.  It lives in mapped, pinned host memory, so
// kernels set it with plain stores and the host reads it without waiting
// for the plan's stream.
struct DevStatus {
  unsigned flags;  // kStatusNonFinite
  int angle;       // an angle whose Fourier error was not finite
};
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusTimeout = 2u;  // a bounded device wait gave up

struct Assembly {
  float2* F = nullptr;        // [Np][N][N] z-transformed spectra, [n][ku][z]
  float2* vol = nullptr;      // [N][N][N] grid, then the centred volume
  int32_t* cell_ptr = nullptr;  // [N*N + 1] CSR rows (cells ky*N + kx)
  int32_t* ent_idx = nullptr;   // sample index n*N + ku
  double* ent_w = nullptr;      // normalised bilinear weight
  double* moments = nullptr;    // [Np][3] sum rho, sum rho*z, sum rho*u
  int64_t n_ent = 0;
  bool ready = false;    // a volume of the current angles may be read
  bool grid_ok = false;  // the gridding lists match the current angles
};

}  // namespace cpra

struct cpra_plan_s {
  cpra_config cfg;
  cudaStream_t stream = nullptr;
  // volume downloads that overlap later work (cpra_assemble_3d_async)
  float2* dl_buf = nullptr;  // staging copy of the volume being downloaded
  cudaStream_t dl_stream = nullptr;
  cudaEvent_t dl_ready = nullptr, dl_done = nullptr;
  bool dl_pending = false;
  // intensity uploads from host memory, on their own stream and buffer, so
  // that they overlap work already queued on the plan's stream
  float* ul_buf = nullptr;  // Np*N*N floats, allocated on the first host upload
  cudaStream_t ul_stream = nullptr;
  cudaEvent_t ul_done = nullptr, ul_free = nullptr;
  bool ul_used = false;  // ul_free has been recorded (the buffer was read)
  int N = 0, Np = 0, W = 0;
  int64_t t = 0;
  bool state_ready = false;
  bool hp_valid = false;
  int n_loaded = 0;
  std::vector<uint8_t> loaded;
  std::vector<double> theta;
  int engine = CPRA_ENGINE_TWO_PASS;

  float* g = nullptr;
  float* g_alt = nullptr;
  float2* Hp = nullptr;
  float* A_main = nullptr;
  float* A_nyq = nullptr;
  double* Cn = nullptr;
  double* sumA2 = nullptr;
  double* err_acc = nullptr;
  uint32_t* S = nullptr;
  double* err_hist = nullptr;
  int64_t err_cap = 0;
  float2* tw = nullptr;        // forward twiddles exp(-2 pi i k/N)
  float2* xtw = nullptr;       // warp-FFT cross twiddles, [k1][l] = exp(-2 pi i l k1/N)
  uint16_t* tcw = nullptr;     // tensor-core DFT matrices (BF16 / FP16 precision)
  float* stage = nullptr;      // staging for host inputs, Np*N*N floats
  uint8_t* bad = nullptr;      // device, Np bytes: 1 where the last load of the angle was invalid
  cpra::DevStatus* status_h = nullptr;  // mapped pinned host memory (cudaHostAlloc)
  cpra::DevStatus* status_d = nullptr;  // its device address
  float* sw_tmp = nullptr;     // shrink-wrap scratch, Np*N*N floats
  unsigned* sw_max = nullptr;  // per-angle max (float bits)
  float* sw_taps = nullptr;    // periodic Gaussian taps
  int sw_ntaps = 0;
  float* po_tmp = nullptr;
  uint8_t* mask = nullptr;     // measured-pixel mask (cpra_load_mask), centred; NULL = all
  bool mask_per_angle = false;
  bool masked = false;         // intensities were loaded under a mask (kernels check A_sym < 0)
  cpra::Assembly asmb;
  // Step C merge scratch (cpra_merge with this plan as destination)
  float2* mg_acc = nullptr;    // [Np][N][N] merged spectra (sums, then the mean)
  float* mg_mag = nullptr;     // [Np][N][N] sums of |E| for the PRTF
  float2* mg_ref = nullptr;    // [N][N] E of the reference PO of the best guess
  double* mg_dist = nullptr;   // [2] twin distances
  float* mg_prtf = nullptr;    // [Np][N/2] PRTF staging for host outputs
  bool merged = false;         // mg_acc holds the mean of the last merge
  // Step D refinement (cpra_refine_3d)
  int vol_state = 0;           // 0 none, 1 Step D volume (assemble or merge), 2 refined
  float2* rf_X = nullptr;
  float2* rf_V = nullptr;
  float* rf_R = nullptr;
  float* rf_B = nullptr;
  uint32_t* rf_S3 = nullptr;
  uint8_t* rf_M = nullptr;
  double* rf_err = nullptr;    // [2 * rf_err_cap] error sums per iteration
  int64_t rf_err_cap = 0;
  double2* rf_cs = nullptr;    // [Np] (cos, sin) of the angles
  int2* rf_shift = nullptr;    // [Np] whole-pixel mass-centre shifts (dz, du)
  float* rf_taps = nullptr;    // [N] periodic Gaussian taps of the last shrink
  unsigned* rf_max = nullptr;
  int64_t rf_t = 0;            // refinement iterations run
  // kernel tables of this plan as a one-job launch
  cpra::JobStatic* d_js = nullptr;
  int2* d_tiles = nullptr;     // (0, angle) of every iterating angle, ascending
  // angles that iterate (cpra_set_present); all of them unless partial
  uint8_t* present = nullptr;  // device, Np bytes
  std::vector<uint8_t> present_h;
  int n_present = 0;
  bool partial = false;
  int64_t present_version = 0;
  cpra::JobStep* d_steps = nullptr;
  int64_t steps_cap = 0;

  // device-time profiling of launches (cpra_set_profiling)
  struct Timed { int kind; cudaEvent_t a, b; };
  bool profiling = false;
  std::vector<Timed> pending;
  std::vector<Timed> spare;
  double kms[CPRA_KERNEL_KINDS] = {0};
  long long kcount[CPRA_KERNEL_KINDS] = {0};

  std::string err;
  std::vector<void*> owned;
};

namespace cpra {

// kernels launched by this library in this process (cpra_launch_count)
extern std::atomic<long long> g_launches;

enum Algo { kHIO = 0, kER = 1, kRAAR = 2 };

// Real-space step of one pixel from the old iterate g, g' = Re IFFT2(P_M G)
// and its support bit.
//   HIO  (Fienup):  g' on V = {in S, g' >= 0}, g - beta g' elsewhere
//   ER:             g' on V, 0 elsewhere
//   RAAR (Luke 2005, T = beta/2 (R_S R_M + I) + (1 - beta) P_M with the
//        reflections R = 2P - I): R_M g = 2g' - g, so g' where 2g' - g lies
//        in the support-positivity set, beta g + (1 - 2 beta) g' elsewhere;
//        c2 = 1 - 2 beta.
template <int ALGO>
__device__ __forceinline__ float update_pixel_t(float g, float gp, bool in_s, float beta, float c2) {
  if constexpr (ALGO == kRAAR) return (in_s && fmaf(2.0f, gp, -g) >= 0.0f) ? gp : fmaf(beta, g, c2 * gp);
  const bool v = in_s && gp >= 0.0f;
  if constexpr (ALGO == kHIO) return v ? gp : fmaf(-beta, gp, g);
  return v ? gp : 0.0f;
}
__device__ __forceinline__ float update_pixel(float g, float gp, bool in_s, int algo, float beta,
                                              float c2) {
  if (algo == kRAAR) return update_pixel_t<kRAAR>(g, gp, in_s, beta, c2);
  if (algo == kHIO) return update_pixel_t<kHIO>(g, gp, in_s, beta, c2);
  return update_pixel_t<kER>(g, gp, in_s, beta, c2);
}

// prepare / state kernels (k_prepare.cu)
cudaError_t launch_prepare(cpra_plan_s* p, const float* I, int first, int count);
cudaError_t launch_support_box(cpra_plan_s* p);
cudaError_t launch_support_u8(cpra_plan_s* p, const uint8_t* S, int per_angle);
cudaError_t launch_init_guess(cpra_plan_s* p);
cudaError_t launch_export_po(cpra_plan_s* p, float* out);
cudaError_t launch_export_support(cpra_plan_s* p, uint8_t* out);
cudaError_t launch_bits_from_u8(uint32_t* bits, const uint8_t* src, int N, int count,
                                cudaStream_t st);
cudaError_t launch_bits_to_u8(const uint32_t* bits, uint8_t* out, int N, int count,
                              cudaStream_t st);

// two-pass iteration (k_twopass.cu, k_fast.cu)
struct CoupleArgs {
  int n_taps;        // 1 = no coupling
  float alpha[CPRA_MAX_TAPS];
  int mirror;
  int object;        // blend P_{S+} g instead of g
  int store_g;       // write the coupled rows to g_dst
  int sweep;         // Gauss-Seidel: taps on angles before n read g_dst
};

// Per-reconstruction pointers and constants, read by the kernels from a
// device table so that one launch can serve many reconstructions.
struct JobStatic {
  float2* Hp;
  const float* A_main;
  const float* A_nyq;
  const double* Cn;
  const double* sumA2;
  double* err_acc;
  const uint32_t* S;
  double* err_hist;
  const float2* tw;
  const float2* xtw;
  const uint16_t* tcw;  // 16-bit block DFT matrices (tensor-core precision)
  const uint8_t* present;  // angles that iterate (coupling renormalises), NULL = all
  DevStatus* status;       // device address of the plan's status word
  int Np, W;
  float beta;
  int pad;
};

// The Fourier error E_F of angle n from its FP64 sums (error terms of the
// column pass + the constant C_n, over sum A^2), as written to the error
// history.  A non-finite sum means a non-finite iterate (a diverged run, a
// NaN or Inf state) or an invalid pattern (the preparation poisons C_n):
// it is flagged in the plan's status word, which the next call reports.
__device__ __forceinline__ double publish_error(double acc, double cn, double den, DevStatus* st,
                                                int n) {
  const double num = acc + cn;
  if (!isfinite(num) || !isfinite(den)) {
    volatile DevStatus* v = st;
    v->angle = n;
    v->flags = kStatusNonFinite;
  }
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

// What one reconstruction does in one iteration (device table, one entry
// per job per iteration).
struct JobStep {
  const float* g_src;  // prime: source stack (coupling reads the neighbours here)
  float* g_dst;        // prime: coupled stack, written when ca.store_g
  float* g;            // the iterate the row pass updates in place
  long long err_slot;  // error-history row, -1 = none
  int prime;           // run the prime kernel (coupling and/or row R2C)
  int algo;            // kHIO / kRAAR / kER; fused engine: the rule of its
                       // first hio_left iterations (ER after them)
  int forward;         // row pass also computes the next row spectra
  int active;          // 0: the column and row passes skip this job
  CoupleArgs ca;
  int n_iters;         // fused engine: iterations of this launch (prime first)
  int hio_left;        // fused engine: how many of them are HIO (the rest ER)
};

// Arguments of the warp engine's persistent work-queue kernel (k_persist_w
// in fast_kernels.cuh).
struct PersistArgs {
  const JobStatic* js;
  const JobStep* st;  // step rows of the call: iteration i of this launch at st + (row0 + i) * m
  const int2* tiles;  // (member, angle) tiles
  int ntiles, m, row0, iters;
  int chunk;          // tiles a chunk: the queue runs chunk by chunk, all iterations each
  unsigned* ticket;   // [2]: next task; [1] is a count that no task increments
  unsigned* done;     // [2 * ntiles]: column and row blocks done in this launch
  long long budget;   // clock64 cycles a wait may take
  int hold;           // testing: the first task waits on ticket[1] >= 1 (never)
};

// One launch over ntiles (job, angle) tiles.
struct Launch {
  int N;
  int engine;
  int prec;  // CPRA_FP32 / CPRA_BF16_TC / CPRA_FP16_TC
  int masked;  // some amplitude carries the missing-data sentinel (A_sym < 0)
  cudaStream_t stream;
  const JobStatic* js;
  const JobStep* st;
  const int2* tiles;
  int ntiles;
};

cudaError_t prepare_kernels(int N, int engine, int prec);  // shared-memory attributes, before capture
cudaError_t launch_prime(const Launch& L);
cudaError_t launch_colpass(const Launch& L);
cudaError_t launch_rowpass(const Launch& L);
cudaError_t launch_shrinkwrap(cpra_plan_s* p);

// assembly (k_assemble.cu)
cudaError_t launch_assemble(cpra_plan_s* p);

// Step C merge (k_assemble.cu): modes of the spectra kernel
enum SpecMode { kSpecF = 0, kSpecRef = 1, kSpecDist = 2, kSpecAcc = 3 };
struct MergeArgs {
  int n0;         // first angle of the launch
  int inv;        // ACC: add conj(E), the spectrum of the centrally inverted PO
  float2* ref;    // REF: E of one PO, [kz][ku] (written); DIST: read
  float2* acc;    // ACC: [Np][kz][ku] += E or conj(E)
  float* mag;     // ACC: [Np][kz][ku] += |E| (NULL = skip)
  double* dist;   // DIST: [0] += sum |ref - E|^2, [1] += sum |ref - conj E|^2
};
// moments of guess g into `moments`, then the spectra kernel in `mode` over
// angles ma.n0 .. ma.n0 + count - 1 (the R2C rows of rho are in g's Hp)
cudaError_t launch_merge_guess(cpra_plan_s* g, double* moments, int mode, const MergeArgs& ma,
                               int count, cudaStream_t st);
// Step D refinement (k_refine.cu): buffers of one plan's refinement
struct RefineArgs {
  int N, W;            // W = ceil(N/32) words per x row of S3
  float2* X;           // [N^3] working spectrum / volume
  float2* V;           // [N^3] gridded spectrum, FFT order
  float* R;            // [N^3] real iterate rho
  float* Bv;           // [N^3] shrink-wrap blur scratch
  uint32_t* S3;        // [N][N][W] 3D support bits
  uint8_t* M;          // [N][N] measured (ky, kx) cells
  const float2* tw;    // twiddles exp(-2 pi i k/N)
  const float2* xtw;   // warp-FFT cross twiddles (N = 64 ... 1024, powers of two)
};
// X = vol (centred), R = Re vol, V = FFT3(X)
cudaError_t launch_refine_setup(const RefineArgs& a, const float2* vol, cudaStream_t st);
// S3 from the 2D supports S2 [Np][N][W] moved by shift[n] = (dz, du), with
// (cos, sin) of every angle; M from the gridding lists
cudaError_t launch_refine_support(const RefineArgs& a, const uint32_t* S2, const double2* cs,
                                  const int2* shift, int Np, const int32_t* cell_ptr, cudaStream_t st);
// FP64 moments (sum rho, sum rho z, sum rho u) of rho = P_{S+} g of every angle
cudaError_t launch_moments(cpra_plan_s* p, double* moments, cudaStream_t st);
// one iteration; err2[0..1] += sum_M |X - V|^2, sum_M |V|^2
cudaError_t launch_refine_iter(const RefineArgs& a, double* err2, cudaStream_t st);
// the same passes with warp-resident FFTs (k_refine_w.cu; fast_supported(N))
cudaError_t launch_refine_fft3_w(const RefineArgs& a, cudaStream_t st);
cudaError_t launch_refine_iter_w(const RefineArgs& a, double* err2, cudaStream_t st);
// S3 <- {blur(P_{S3+} R) >= tau max} (mx: one unsigned of scratch)
cudaError_t launch_refine_shrink(const RefineArgs& a, const float* taps, int ntaps, float tau,
                                 unsigned* mx, cudaStream_t st);
// vol = P_{S3+} R
cudaError_t launch_refine_output(const RefineArgs& a, float2* vol, cudaStream_t st);

// PRTF (prtf != NULL, needs mag), acc <- acc / n_l, its IDFT_z into dst's F,
// gridding and the plane IFFTs into dst's volume, on dst's stream
cudaError_t launch_merge_finish(cpra_plan_s* dst, float2* acc, const float* mag, float* prtf,
                                int n_l);

bool n_supported(int N);

// two-pass engine with warp-resident FFTs (k_fast.cu)
bool fast_supported(int N);          // iteration kernels (WARP engine)
bool refine_fast_supported(int N);   // 3D refinement passes and tensor-core forms
bool fast_dims(int N, int* E1, int* E2);
cudaError_t prepare_kernels_fast(int N);
cudaError_t prepare_kernels_fast_tc(int N, int prec);
cudaError_t launch_rowpass_fast_tc(const Launch& L);
cudaError_t launch_prime_fast_tc(const Launch& L);
cudaError_t launch_colpass_fast_tc(const Launch& L);
cudaError_t launch_rowpass_fast(const Launch& L);
cudaError_t launch_prime_fast(const Launch& L);
cudaError_t launch_colpass_fast(const Launch& L);
// persistent work-queue form of the column and row passes (FP32)
bool persist_supported(int N);
cudaError_t prepare_persist(int N, int* blocks_per_sm);
cudaError_t launch_persist(int N, const PersistArgs& a, int masked, int grid, cudaStream_t st);

// cluster-resident fused engine (k_fused.cu): one launch = prime + n_iters
// iterations of every tile, the angle's spectrum held in distributed shared
// memory
bool fused_supported(int N);
cudaError_t prepare_kernels_fused(int N);
cudaError_t launch_fused(const Launch& L);

// records a failure of a call without a plan (cpra_last_error(NULL))
cpra_status record_error(cpra_status st, const std::string& msg);

}  // namespace cpra
