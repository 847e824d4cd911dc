// Shared device/host definitions of the DDI library: the plan object, complex helpers,
// error reporting.  Included by every .cu translation unit of the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/ddi.h"
#include "tables.h"

namespace ddi {

// ---- error reporting (thread-local message behind ddi_last_error) ----------------
void set_error(const char* fmt, ...);
const char* last_error();

#define DDI_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ::ddi::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                       __LINE__);                                                       \
      return DDI_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

#define DDI_LAUNCH_CHECK()                                                              \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) {                                                            \
      ::ddi::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),      \
                       __FILE__, __LINE__);                                             \
      return DDI_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

// Runs f() (returning a status) so that no C++ exception crosses the C ABI: a failed host
// allocation becomes DDI_ERR_OOM, any other exception DDI_ERR_INTERNAL, with the message
// kept for ddi_last_error().
template <typename F>
int guarded(const char* where, F&& f) noexcept {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    set_error("%s: host allocation failed", where);
    return DDI_ERR_OOM;
  } catch (const std::exception& e) {
    set_error("%s: %s", where, e.what());
    return DDI_ERR_INTERNAL;
  } catch (...) {
    set_error("%s: unknown exception", where);
    return DDI_ERR_INTERNAL;
  }
}

#define DDI_TRY(expr)          \
  do {                         \
    int s_ = (expr);           \
    if (s_ != DDI_OK) return s_; \
  } while (0)

// ---- complex types -------------------------------------------------------------
template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) {
  C r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }

// ---- spread work list ------------------------------------------------------------
struct SpreadUnit {
  int tile;   // linear tile index (tz * ntiles_y + ty) * ntiles_x + tx
  int plane;  // owned z-plane of the tile in 3D; 0 in 2D (the unit is the whole tile)
  int lo, hi; // range of visit-list entries whose taps cover the plane
  int slot;   // -1: write the plane to the fine grid; >= 0: write to partial slot
};
struct SplitUnit {
  int tile, plane, slot0, nslots;
};

// ---- column spread work list (FP32 3D) -------------------------------------------------------
// A column is a kColX x kColY block of fine cells in x-y with all its z-planes.  A work unit
// takes a range of the column's visits, sorted by their first z tap, and a window of planes.
constexpr int kColX = 8, kColY = 8;
struct ColUnit {
  int col;       // column index cy * (nf_x / kColX) + cx
  int lo, hi;    // visit range
  int z0, z1;    // planes [z0, z1) the unit writes (plane z mod nf_z; z1 may exceed nf_z)
  int plo, phi;  // leading / trailing planes that other units also touch: go to partial slots
  int slot0;     // its shared planes (leading, then trailing) are entries slot0 .. of the unit slot map
};
struct alignas(16) ColRed {  // a plane of a column touched by several units: the sum of their partial slots
  int col, z;
  int s0, ns;    // partial slots [s0, s0 + ns), one per unit touching the plane, in unit order
};

// ---- spread tile geometry (host and device) -------------------------------------------------
constexpr int kSpreadThreads = 128;  // 4 warps per CTA, each taking work units on its own

// first fine cell of tile t along an axis: t T - T/2 (mod nf), i.e. the tile lattice is
// shifted by half a tile so that k = 0 lies inside a tile; unshifted with a single tile
__host__ __device__ inline int tile_origin(int t, int T, int ntile, int nf) {
  if (ntile == 1) return 0;
  const int o = t * T - T / 2;
  return o < 0 ? o + nf : o;
}
// start of a footprint relative to a tile origin: l0 - T0 wrapped into [-(w-1), nf-(w-1)),
// so that footprints reaching the tile from below through the periodic wrap are negative
__host__ __device__ inline int rel_start(int l0, int T0, int nf, int w) {
  int o = l0 - T0;
  if (o < 0) o += nf;
  if (o > nf - w) o -= nf;
  return o;
}
// Row stride (cells) of the spread's shared-memory plane.  A warp touches 4 rows of 8
// consecutive cells (8-byte cells: half the 128-byte bank window each); with a stride of
// 8 (mod 16) cells consecutive rows fall in opposite halves, so the 32 accesses take the
// minimum two wavefronts.  (16-byte cells fill the window with one 8-cell row segment.)
__host__ __device__ inline int spread_row_stride(int TX) { return TX + ((8 - TX % 16) + 16) % 16; }

// a processed node's symbol direction (x, y, z; 2D: cos, sin, 0) and weight without the
// symbol, FP64, from which its weight is rebuilt for other dipole axes
struct alignas(16) NodeDir {
  double x, y, z, w;
};

// ---- the plan ----------------------------------------------------------------------
struct Plan {
  ddi_plan_desc desc{};
  int dim = 3, prec = DDI_FP64;
  int n[3] = {1, 1, 1};
  int nf[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  double dv = 1.0;  // h_1 h_2 h_3
  int w = 8;
  double beta = 0.0;
  int64_t M = 0, Mh = 0;
  int tile[3] = {1, 1, 1};
  int ntile[3] = {1, 1, 1};
  int chunk = 0;
  int device = 0;
  size_t bytes = 0;

  QuadTables quad;                   // host copy of the tables (export, tests)
  std::vector<int64_t> order;        // processing order -> original node index
  std::vector<ushort4> h_l0;         // host copy of d_l0 (spread lists are rebuilt from it)
  std::vector<int> h_zcls;           // z class of each processed node (equal first z tap and psi_z row)
  bool gpe_ready = false;            // GPE workspace allocated (plans of a batch have none)
  size_t spread_bytes = 0;           // device bytes of the spread lists and partial planes
  double tuned_ms = 0.0;             // spread time of the tile the autotuner chose (0: not tuned)

  // device arrays (element types depend on prec), nodes in processing order
  void* d_l0 = nullptr;       // ushort4 [Mh]: wrapped first tap (x, y, z)
  void* d_psi = nullptr;      // T [Mh][3][w]: kernel values along x, y, z at the w taps
  void* d_scale = nullptr;    // T [Mh]: 2 h^d W_q
  NodeDir* d_dirw = nullptr;  // [Mh]: direction and weight without the symbol (ddi_plan_set_axes)
  void* d_c = nullptr;        // cx [Mh]: node values c_q
  void* d_deconv = nullptr;   // double [n0 + n1 + n2]: 1/psihat per axis, index j (0..n-1)
  void* d_deconv_x2 = nullptr;  // float2 [n0]: the x factors as FP32 head + tail (FP32 plans)
  void* d_ones = nullptr;     // double [n0 + n1 + n2] of ones: the pad and crop of a split plan's smooth part
  void* d_ones_x2 = nullptr;  // float2 [n0] of (1, 0)
  void* d_fine = nullptr;     // cx [nf0 nf1 nf2]
  void* d_partial = nullptr;  // cx [nslots * tile cells]
  int4* d_visits = nullptr;   // spread visit lists: (node, ox, oy, oz) relative to the tile
  SpreadUnit* d_units = nullptr;
  SplitUnit* d_split = nullptr;
  int* d_counter = nullptr;   // unit counter of the persistent spread
  int* d_nonfinite = nullptr; // set by the pad pass when rho holds NaN / Inf (cleared by checks)
  // column spread (spread_kind == DDI_SPREAD_COLUMNS)
  int spread_kind = DDI_SPREAD_TILES;
  int2* d_cvis = nullptr;     // visits (node, first z tap << 13 | z-class start << 12 | (oy + 16) << 6 | (ox + 16))
  ColUnit* d_cunits = nullptr;
  ColRed* d_cred = nullptr;
  int* d_cslots = nullptr;    // per unit (from its slot0): the partial slot of each shared plane
  
  void* d_cpart = nullptr;    // partial planes: [slot][kColY * kColX] complex
  int ncunits = 0, ncred = 0, ncslots = 0;
  bool col_comp = false;      // column spread: compensated (Kahan) plane accumulation
  long long visits = 0;       // total visit-list entries
  long long pairs = 0;        // total (node, plane) pairs of all units
  int npl = 1;                // owned planes per tile (z-planes in 3D; 1 in 2D)
  int nunits = 0;
  size_t spread_smem = 0;     // launch geometry of the spread (fixed per plan)
  int spread_blocks = 1;
  int nsplit = 0, nslots = 0;
  // split plans: half-widths of the band of fine-grid lines around k = 0 that hold every tap
  // of the ball's nodes (x and y; 0 = all lines); the ball's NUFFT passes skip the others
  int band[2] = {0, 0};
  // fine-grid y lines that hold node taps: yr[0], yr[0] + 1, .. (mod nf_y), yr[1] of them;
  // the NUFFT's z passes transform only these columns and its y passes only store / read them
  int yr[2] = {0, 1};
  // fine-grid x lines that hold node taps (every line, except for split plans' ball band)
  int xr[2] = {0, 1};
  bool precise_nufft = false;  // NUFFT passes apply FP32 twiddles as head + tail
  bool batch_item = false;     // built by ddi_batch_create (2D items spread by columns, see create_plan)
  int tw_n[8] = {};           // lengths of the twiddle tables below
  void* d_tw[8] = {};         // cx twiddle tables e^{-2 pi i k / n} (FP32: n heads, then n tails)
  // GPE workspace
  void* d_psi1 = nullptr;     // cx [N]
  void* d_rho = nullptr;      // T [N]
  void* d_phi = nullptr;      // T [N]
  void* d_work = nullptr;     // cx [N]
  void* d_work2 = nullptr;    // cx [N]
  void* d_kin = nullptr;      // cx [n0 + n1 + n2]: per-axis kinetic phase factors
  double* d_red = nullptr;    // reduction partials
  double* h_red = nullptr;    // pinned host copy of reduction results
  void* d_io_in = nullptr;    // staging for ddi_apply_host
  void* d_io_out = nullptr;
  int red_blocks = 0;

  // per-launch CUDA events for ddi_apply_timed (recorded only while `timing` is set)
  bool timing = false;
  int nmarks = 0;
  const char* mark_names[64] = {};
  cudaEvent_t mark_ev[65] = {};
  bool ev_created = false;
  void mark(const char* name, cudaStream_t s) {
    if (!timing || nmarks >= 64) return;
    mark_names[nmarks] = name;
    cudaEventRecord(mark_ev[nmarks + 1], s);
    ++nmarks;
  }

  // the improved split algorithm (Eq. 3.9): the nodes are the small ball's, and the smooth
  // part is added by a padded FFT convolution
  bool split() const { return desc.split_k0 > 0.0; }
  int64_t grid_points() const { return (int64_t)n[0] * n[1] * n[2]; }
  // cells of one owned plane's shared-memory buffer (padded row stride)
  size_t spread_plane_cells() const { return (size_t)tile[1] * spread_row_stride(tile[0]); }
  int64_t fine_points() const { return (int64_t)nf[0] * nf[1] * nf[2]; }
  size_t real_size() const { return prec == DDI_FP64 ? 8 : 4; }
  size_t cx_size() const { return prec == DDI_FP64 ? 16 : 8; }
};

inline const void* twiddles(const Plan& p, int n) {
  for (int i = 0; i < 8; ++i)
    if (p.tw_n[i] == n) return p.d_tw[i];
  return nullptr;
}

// ---- FFT (fft.cu) ------------------------------------------------------------------
// In-place batched 1-D FFTs along one axis of a [nz][ny][nx] complex array, unnormalised,
// dir = -1: e^{-2 pi i jk/n}, dir = +1: e^{+2 pi i jk/n}.  axis 0 = x, 1 = y, 2 = z.
template <typename T>
int fft_axis(const Plan& p, cx_t<T>* data, int nx, int ny, int nz, int axis, int dir, cudaStream_t s);
template <typename T>
int fft_3d(const Plan& p, cx_t<T>* data, int nx, int ny, int nz, int dir, cudaStream_t s);
int make_twiddles(Plan& p, int n);

// ---- pruned / fused fine-grid FFTs of the NUFFT (fft_nufft.cu) ----------------------
template <typename T> int nufft_forward_fft(Plan& p, const T* rho, cudaStream_t s);  // rho -> F (fine grid)
// U (fine grid) -> phi; acc: phi += the result instead of phi = the result
template <typename T> int nufft_inverse_fft(Plan& p, T* phi, cudaStream_t s, bool acc = false);
// split plans: phi = I_1 of Eq. 3.9 (zero-padded FFT convolution of rho with the smooth
// symbol p = (1 - q) Uhat on the fine grid); reads rho before it writes phi (they may alias)
template <typename T> int split_smooth_part(Plan& p, const T* rho, T* phi, cudaStream_t s);

// ---- NUFFT stages (nufft.cu) --------------------------------------------------------
template <typename T> int run_type2(Plan& p, const T* rho, cudaStream_t s);         // rho -> d_c
template <typename T> int run_type1_from_c(Plan& p, T* phi, cudaStream_t s);       // d_c -> phi
template <typename T> int run_ddi(Plan& p, const T* rho, T* phi, cudaStream_t s);
// bytes of the spread's per-warp node stage of 32 nodes: psi_x and psi_y rows (psi_y padded
// to the lanes' row groups) and a 16-byte (FP32) / 32-byte (FP64) header per node
__host__ __device__ constexpr int spread_rows_per_instr(int w) { return 32 / (w <= 8 ? 8 : 16); }
__host__ __device__ constexpr size_t spread_stage_bytes(int w, size_t real_bytes) {
  return 32 * (size_t)w * real_bytes +
         32 * (size_t)(((w + spread_rows_per_instr(w) - 1) / spread_rows_per_instr(w)) * spread_rows_per_instr(w)) *
             real_bytes +
         32 * (real_bytes == 4 ? 16 : 32);
}
// shared memory of one spread warp: its plane buffer and its node stage, 16-byte aligned
__host__ __device__ inline size_t spread_warp_bytes(size_t plane_bytes, size_t stage_bytes) {
  return ((plane_bytes + 15) & ~(size_t)15) + ((stage_bytes + 15) & ~(size_t)15);
}

int configure_kernels(Plan& p);  // per-plan launch geometry (nufft.cu)
// reads and clears the plan's non-finite-input record after synchronising s:
// DDI_ERR_NONFINITE if it was set (plan.cu)
int take_nonfinite(Plan& p, cudaStream_t s);

// ---- plans (plan.cu) ------------------------------------------------------------------------
int create_plan(Plan& p, const ddi_plan_desc* desc, cudaStream_t stream, bool gpe = true, bool batch_item = false);
void set_tile(Plan& p, const int want[3]);         // tile rounded as for ddi_plan_desc.tile
int build_spread(Plan& p, cudaStream_t stream);     // spread lists for the current tile
int build_spread_col(Plan& p, cudaStream_t stream); // column spread lists for desc.chunk (plan.cu)
bool columns_apply(const Plan& p);                   // the column spread fits the plan (plan.cu)
void drop_spread_lists(Plan& p);                    // frees both schemes' spread lists (plan.cu)
int time_spread(Plan& p, cudaStream_t s, int reps, float* ms);  // best of reps (nufft.cu)
int tune_spread_tile(Plan& p, cudaStream_t s);      // autotuner (batch.cu)
void destroy_plan(Plan& p);
void fill_info(const Plan& p, ddi_plan_info* info);
int set_axes(Plan& p, const double* axis_n, const double* axis_m, cudaStream_t s);  // (plan.cu)

}  // namespace ddi

struct ddi_plan_s {
  ddi::Plan p;
};
