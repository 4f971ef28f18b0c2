// C ABI of libgcdf (include/gcdf.h): argument checks, net construction
// (weight layouts for each path), temporaries and launch sequence.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gcdf_internal.cuh"

using namespace gcdf;

namespace gcdf {
cudaError_t launch_project(const float* q, int N, int n, const int* offsets, int M, long long K, const float* f,
                           const float* m_diag, float* g, cudaStream_t s);
int fp32_tile_pairs(int H);
int tc_tile_pairs();
bool tc_supported(int H, int L, int n_dof);
}  // namespace gcdf

namespace {
constexpr int kSmemLimit = 227 * 1024 - 1024;  // per-block opt-in limit less static shared memory
}

struct gcdf_net {
  int n_dof, H, L, precision, d_q, d_in;
  int device, num_sms;
  float* w_dev;      // original FP32 weights (layout of gcdf_weight_count)
  // FP32 path images
  float* BF;
  float* BB;
  float* bias_p;
  float* wout_p;
  // BF16 tensor-core path images
  uint16_t* slabs;   // 16-bit operand image (BF16 or FP16 bits)
  float* tc_bias;
  float* tc_w1p;
  TcWeights tcw;     // tensor maps and pointers for the tensor-core kernel
  int* err_word;     // device status word written by bounded waits
  int active_set;    // HINGE / MIN: value-only pass, then gradients of the active pairs only
  float bout;
  size_t off_W1, off_b1, off_wout;
  cudaEvent_t prof_start, prof_stop;  // optional events around the fused kernel
};

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? GCDF_ENOMEM : GCDF_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int shape_check(const gcdf_net_desc* d) {
  if (!d) return fail(GCDF_EINVAL, "desc is NULL");
  if (d->n_dof < 3 || d->n_dof > kMaxDof) return fail(GCDF_EINVAL, "n_dof %d outside [3, %d]", d->n_dof, kMaxDof);
  if (d->n_hidden_layers < 2) return fail(GCDF_EINVAL, "n_hidden_layers %d < 2", d->n_hidden_layers);
  if (d->precision != GCDF_FP32 && d->precision != GCDF_BF16 && d->precision != GCDF_FP16 && d->precision != GCDF_FP8)
    return fail(GCDF_EINVAL, "unknown precision %d", d->precision);
  if (d->hidden <= 0 || d->hidden > 512 || d->hidden % 32)
    return fail(GCDF_EINVAL, "hidden %d must be a positive multiple of 32, at most 512", d->hidden);
  return GCDF_OK;
}

size_t weight_count(int n_dof, int H, int L) {
  const size_t d_in = 3 + 2 + 2 * (size_t)(n_dof - 2);
  return H * d_in + H + (size_t)(L - 1) * ((size_t)H * H + H) + H + 1;
}

template <class T>
int dev_alloc_copy(T** dst, const T* src, size_t count) {
  cudaError_t e = cudaMalloc((void**)dst, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return GCDF_OK;
}

// Column permutation of the FP32 path's biases and w_o: feature c = fg + G f
// -> column 8 fg + f (a thread's 8 features are 8 consecutive floats).
inline int perm_col(int c, int H) {
  const int G = H / 8;
  return (c % G) * 8 + c / G;
}
// Column permutation of its weight images: feature c = fg + G f -> column
// 4 fg + f (f < 4) or H / 2 + 4 fg + f - 4, so that the 8 feature groups of a
// warp read their first and their second four features of a row as two
// contiguous 128-byte pieces.
inline int perm_wcol(int c, int H) {
  const int G = H / 8, fg = c % G, f = c / G;
  return f < 4 ? 4 * fg + f : H / 2 + 4 * fg + f - 4;
}

int build_fp32_images(gcdf_net* net, const float* w) {
  const int H = net->H, L = net->L;
  std::vector<float> BF((size_t)(L - 1) * H * H), BB((size_t)(L - 1) * H * H);
  std::vector<float> bias((size_t)(L - 1) * H), wout(H);
  size_t off = (size_t)H * net->d_in + H;
  for (int l = 0; l < L - 1; ++l) {
    const float* W = w + off;
    const float* b = W + (size_t)H * H;
    for (int o = 0; o < H; ++o) {
      for (int i = 0; i < H; ++i) {
        const float v = W[(size_t)o * H + i];
        BF[(size_t)l * H * H + (size_t)i * H + perm_wcol(o, H)] = v;  // row = input, col = output
        BB[(size_t)l * H * H + (size_t)o * H + perm_wcol(i, H)] = v;  // row = output, col = input
      }
      bias[(size_t)l * H + perm_col(o, H)] = b[o];
    }
    off += (size_t)H * H + H;
  }
  for (int c = 0; c < H; ++c) wout[perm_col(c, H)] = w[off + c];
  int rc;
  if ((rc = dev_alloc_copy(&net->BF, BF.data(), BF.size()))) return rc;
  if ((rc = dev_alloc_copy(&net->BB, BB.data(), BB.size()))) return rc;
  if ((rc = dev_alloc_copy(&net->bias_p, bias.data(), bias.size()))) return rc;
  if ((rc = dev_alloc_copy(&net->wout_p, wout.data(), wout.size()))) return rc;
  return GCDF_OK;
}

int build_tc_images(gcdf_net* net, const float* w) {
  const int H = net->H, L = net->L;
  const int fmt = net->precision == GCDF_FP8 ? 2 : (net->precision == GCDF_FP16 ? 1 : 0);
  // 16-bit elements (FP8 uses the first half of the same buffer)
  std::vector<uint16_t> image(tc_image_elems(H, L, net->d_q));
  memset(net->tcw.fp8_scale, 0, sizeof(net->tcw.fp8_scale));
  tc_build_image(w, H, L, net->d_q, net->d_in, fmt, image.data(), net->tcw.fp8_scale);
  std::vector<float> bias((size_t)(L - 1) * H), w1p((size_t)H * 3);
  size_t off = (size_t)H * net->d_in + H;
  for (int l = 0; l < L - 1; ++l) {
    memcpy(&bias[(size_t)l * H], w + off + (size_t)H * H, H * sizeof(float));
    off += (size_t)H * H + H;
  }
  for (int c = 0; c < H; ++c)
    for (int d = 0; d < 3; ++d) w1p[(size_t)c * 3 + d] = w[(size_t)c * net->d_in + d];
  int rc;
  if ((rc = dev_alloc_copy(&net->slabs, image.data(), image.size()))) return rc;
  if ((rc = dev_alloc_copy(&net->tc_bias, bias.data(), bias.size()))) return rc;
  if ((rc = dev_alloc_copy(&net->tc_w1p, w1p.data(), w1p.size()))) return rc;
  TcWeights& tw = net->tcw;
  if (tc_encode_maps(net->slabs, H, L, net->d_q, fmt, tw)) return fail(GCDF_ECUDA, "cuTensorMapEncodeTiled failed");
  tw.fmt = fmt;
  tw.bias = net->tc_bias;
  tw.W1p = net->tc_w1p;
  tw.wout = net->w_dev + net->off_wout;
  tw.bout = net->bout;
  tw.H = H;
  tw.L = L;
  tw.d_q = net->d_q;
  tw.nj = tc_nj(net->d_q);
  tw.err = net->err_word;
  return GCDF_OK;
}

void free_net(gcdf_net* n) {
  if (!n) return;
  cudaFree(n->w_dev);
  cudaFree(n->BF);
  cudaFree(n->BB);
  cudaFree(n->bias_p);
  cudaFree(n->wout_p);
  cudaFree(n->slabs);
  cudaFree(n->tc_bias);
  cudaFree(n->tc_w1p);
  cudaFree(n->err_word);
  delete n;
}

// Common validation of the per-call arrays.  Returns GCDF_OK and fills `w`.
int check_call(gcdf_net* net, const float* q, int N, const float* p, int M, const int* offsets,
               const int* idx, int n_pairs, const float* shift, WorkDesc& w) {
  if (!net) return fail(GCDF_EINVAL, "net is NULL");
  if (N < 0 || M < 0) return fail(GCDF_EINVAL, "negative size (n_waypoints %d, n_points %d)", N, M);
  if ((offsets == nullptr) != (idx == nullptr))
    return fail(GCDF_EINVAL, "part_offsets and part_idx must both be NULL or both be set");
  long long P = offsets ? (long long)n_pairs : (long long)N * M;
  if (offsets && n_pairs < 0) return fail(GCDF_EINVAL, "n_pairs %d < 0", n_pairs);
  if (P > 0x7fffffffLL) return fail(GCDF_EINVAL, "pair count %lld exceeds 2^31-1", P);
  if (N > 0 && (!q || !aligned16(q))) return fail(GCDF_EINVAL, "q is NULL or not 16-byte aligned");
  if (P > 0 && M > 0 && (!p || !aligned16(p))) return fail(GCDF_EINVAL, "p is NULL or not 16-byte aligned");
  if (offsets && (!aligned16(offsets) || (n_pairs > 0 && !aligned16(idx))))
    return fail(GCDF_EINVAL, "part_offsets / part_idx not 16-byte aligned");
  if (shift && !aligned16(shift)) return fail(GCDF_EINVAL, "shift not 16-byte aligned");
  if (offsets && n_pairs > 0 && M == 0) return fail(GCDF_EINVAL, "point lists given but n_points == 0");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != net->device) return fail(GCDF_EINVAL, "net belongs to device %d, current device is %d", net->device, dev);
  memset(&w, 0, sizeof(w));
  w.q = q;
  w.p = p;
  w.offsets = offsets;
  w.idx = idx;
  w.N = N;
  w.M = M;
  w.n_pairs = (int)P;
  w.n_dof = net->n_dof;
  w.n_ang = net->n_dof - 2;
  w.tile = net->precision == GCDF_FP32 ? fp32_tile_pairs(net->H) : tc_tile_pairs();
  if (offsets) {
    w.tiles_per_wp = 0;
    w.n_tiles = (int)(((long long)n_pairs + w.tile - 1) / w.tile + N);
  } else {
    w.tiles_per_wp = (M + w.tile - 1) / w.tile;
    w.n_tiles = w.tiles_per_wp * N;
  }
  return GCDF_OK;
}

struct Temps {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Temps(cudaStream_t st) : s(st) {}
  cudaError_t get(void** out, size_t bytes) {
    cudaError_t e = lib_malloc_async(out, bytes < 16 ? 16 : bytes, s);
    if (e == cudaSuccess) ptrs.push_back(*out);
    return e;
  }
  ~Temps() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

int run(gcdf_net* net, WorkDesc& w, const float* shift, Temps& tmp, cudaStream_t s) {
  cudaError_t e;
  float *A = nullptr, *trig = nullptr;
  if ((e = tmp.get((void**)&A, (size_t)w.N * net->H * sizeof(float)))) return cuda_fail(e, "cudaMallocAsync");
  if ((e = tmp.get((void**)&trig, (size_t)w.N * 2 * w.n_ang * sizeof(float)))) return cuda_fail(e, "cudaMallocAsync");
  w.A = A;
  w.trig = trig;
  if (w.offsets) {
    int* ts = nullptr;
    if ((e = tmp.get((void**)&ts, (size_t)(w.N + 1) * sizeof(int)))) return cuda_fail(e, "cudaMallocAsync");
    if ((e = launch_tile_map(w.offsets, w.N, w.tile, ts, s))) return cuda_fail(e, "tile map launch");
    w.tile_start = ts;
  }
  if ((e = launch_prep(w, net->w_dev + net->off_W1, net->w_dev + net->off_b1, net->H, net->d_in, shift, A, trig, s)))
    return cuda_fail(e, "prep launch");
  if (net->prof_start && (e = cudaEventRecord(net->prof_start, s))) return cuda_fail(e, "cudaEventRecord");
  if (net->precision == GCDF_FP32) {
    Fp32Weights fw;
    fw.BF = net->BF;
    fw.BB = net->BB;
    fw.bias = net->bias_p;
    fw.W1 = net->w_dev + net->off_W1;
    fw.wout = net->wout_p;
    fw.bout = net->bout;
    fw.H = net->H;
    fw.L = net->L;
    fw.d_in = net->d_in;
    fw.d_q = net->d_q;
    if ((e = launch_fp32(w, fw, net->num_sms, s))) return cuda_fail(e, "fp32 kernel launch");
  } else {
    if ((e = launch_tc(w, net->tcw, net->num_sms, s))) return cuda_fail(e, "tensor-core kernel launch");
  }
  if (net->prof_stop && (e = cudaEventRecord(net->prof_stop, s))) return cuda_fail(e, "cudaEventRecord");
  return GCDF_OK;
}

// HINGE / MIN in two passes: f of every pair (value-only, no reverse sweep),
// the per-waypoint active lists (support.cu), then the fused value + gradient
// pass over those lists alone.  The merge of the second pass gives the cost,
// gradient and argmin of the full reduction (the pairs left out add exactly
// zero); only the order of the HINGE sums differs from the one-pass result.
int reduce_active(gcdf_net* net, WorkDesc& w, const float* shift, float* cost, float* grad, int* argmin,
                  cudaStream_t s) {
  Temps tmp(s);
  cudaError_t e;
  float* fv = nullptr;
  int *cnt = nullptr, *nact = nullptr, *amin = nullptr, *off2 = nullptr, *idx2 = nullptr;
  const size_t cap = w.mode == kHinge ? (size_t)w.n_pairs : (size_t)w.N;
  if ((e = tmp.get((void**)&fv, (size_t)w.n_pairs * sizeof(float))) ||
      (e = tmp.get((void**)&cnt, (size_t)w.N * sizeof(int))) || (e = tmp.get((void**)&nact, (size_t)w.N * sizeof(int))) ||
      (e = tmp.get((void**)&amin, (size_t)w.N * sizeof(int))) ||
      (e = tmp.get((void**)&off2, (size_t)(w.N + 1) * sizeof(int))) || (e = tmp.get((void**)&idx2, cap * sizeof(int))))
    return cuda_fail(e, "cudaMallocAsync");
  // pass 1: every pair's value
  WorkDesc w1 = w;
  w1.mode = kQuery;
  w1.f_out = fv;
  w1.g_out = nullptr;
  int rc = run(net, w1, shift, tmp, s);
  if (rc) return rc;
  if ((e = launch_active_lists(w, fv, cnt, nact, amin, off2, idx2, s))) return cuda_fail(e, "active-list launch");
  // pass 2: value + gradient over the active lists (an upper bound of their
  // length sizes the tiles and records; the kernels read the exact count)
  WorkDesc w2 = w;
  w2.offsets = off2;
  w2.idx = idx2;
  w2.point_base = nullptr;
  w2.tile_start = nullptr;
  w2.tiles_per_wp = 0;
  w2.n_pairs = (int)cap;
  w2.n_tiles = (int)(((long long)cap + w2.tile - 1) / w2.tile + w.N);
  Partial* parts = nullptr;
  if ((e = tmp.get((void**)&parts, (size_t)w2.n_tiles * sizeof(Partial)))) return cuda_fail(e, "cudaMallocAsync");
  w2.partials = parts;
  if ((rc = run(net, w2, shift, tmp, s))) return rc;
  if ((e = launch_merge(w2, w2.N, cost, grad, argmin, s))) return cuda_fail(e, "merge launch");
  return GCDF_OK;
}

// Fused pass plus per-waypoint merge for a validated WorkDesc (mode, param set).
int reduce_call(gcdf_net* net, WorkDesc& w, const float* shift, float* cost, float* grad, int* argmin,
                cudaStream_t s) {
  if (net->active_set && w.n_pairs > 0 && (w.mode == kHinge || w.mode == kMin))
    return reduce_active(net, w, shift, cost, grad, argmin, s);
  Temps tmp(s);
  cudaError_t e;
  Partial* parts = nullptr;
  if ((e = tmp.get((void**)&parts, (size_t)(w.n_tiles > 0 ? w.n_tiles : 1) * sizeof(Partial))))
    return cuda_fail(e, "cudaMallocAsync");
  w.partials = parts;
  if (w.n_pairs > 0) {
    const int rc = run(net, w, shift, tmp, s);
    if (rc) return rc;
  } else if (w.offsets) {
    // every list is empty: the merge sees no tiles
    int* ts = nullptr;
    if ((e = tmp.get((void**)&ts, (size_t)(w.N + 1) * sizeof(int)))) return cuda_fail(e, "cudaMallocAsync");
    if ((e = launch_tile_map(w.offsets, w.N, w.tile, ts, s))) return cuda_fail(e, "tile map launch");
    w.tile_start = ts;
  } else {
    w.tiles_per_wp = 0;
  }
  if ((e = launch_merge(w, w.N, cost, grad, argmin, s))) return cuda_fail(e, "merge launch");
  return GCDF_OK;
}

}  // namespace

namespace gcdf {

// The temporaries of every call come from one memory pool per device owned by
// the library, with no release threshold: memory freed at the end of a call
// stays in the pool for the next one instead of going back to the driver at
// the next synchronisation, which made every call pay for fresh mappings
// (measured: ~90 us of host time per collision-cost call with the device's
// default pool, against ~8 us for the same launches without allocations).
// gcdf_release_cached_memory trims it.
namespace {
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[64] = {};

cudaError_t device_pool(int dev, cudaMemPool_t* out, bool fresh) {
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (fresh && g_pools[dev]) g_pools[dev] = nullptr;  // the context was torn down and recreated
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t lib_malloc_async(void** out, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaMallocAsync(out, bytes, s);
  cudaMemPool_t pool = nullptr;
  if ((e = device_pool(dev, &pool, false)) != cudaSuccess) return e;
  e = cudaMallocFromPoolAsync(out, bytes, pool, s);
  if (e == cudaErrorInvalidValue || e == cudaErrorContextIsDestroyed || e == cudaErrorInvalidResourceHandle) {
    cudaGetLastError();  // clear, then once more with a pool of the current context
    if ((e = device_pool(dev, &pool, true)) != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync(out, bytes, pool, s);
  }
  return e;
}

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = 0; }

int net_n_dof(const gcdf_net* net) { return net->n_dof; }
int net_device(const gcdf_net* net) { return net->device; }

// Device temporaries of the fused pass per waypoint row with M points: the
// first-layer term, the sines and cosines, the tile prefix and the partial
// records of its tiles.
size_t net_step_bytes_per_row(const gcdf_net* net, int M) {
  const int tile = net->precision == GCDF_FP32 ? fp32_tile_pairs(net->H) : tc_tile_pairs();
  const size_t tiles = (size_t)(M + tile - 1) / tile + 1;
  // + with active sets: every pair's value, its list entry, the per-row
  // counters and a second set of tile records
  const size_t act = net->active_set ? (size_t)M * 8 + 20 + tiles * sizeof(Partial) : 0;
  return (size_t)net->H * 4 + (size_t)2 * (net->n_dof - 2) * 4 + 4 + tiles * sizeof(Partial) + act;
}

// Collision cost over range lists: waypoint i uses points point_base[i] ..
// point_base[i] + (offsets[i+1] - offsets[i]) - 1 of p (no index array), or,
// with idx, the CSR lists offsets / idx.
int collision_ranges(gcdf_net* net, const float* q, int N, const float* p, int M, const int* offsets,
                     const int* point_base, const int* idx, int n_pairs, int reduction, float param, float* cost,
                     float* grad, cudaStream_t s) {
  if (N == 0) return GCDF_OK;
  WorkDesc w;
  memset(&w, 0, sizeof(w));
  w.q = q;
  w.p = p;
  w.offsets = offsets;
  w.idx = idx;
  w.point_base = idx ? nullptr : point_base;
  w.N = N;
  w.M = M;
  w.n_pairs = n_pairs;
  w.n_dof = net->n_dof;
  w.n_ang = net->n_dof - 2;
  w.tile = net->precision == GCDF_FP32 ? fp32_tile_pairs(net->H) : tc_tile_pairs();
  w.n_tiles = (int)(((long long)n_pairs + w.tile - 1) / w.tile + N);
  w.mode = reduction;
  w.param = param;
  return reduce_call(net, w, nullptr, cost, grad, nullptr, s);
}

}  // namespace gcdf

extern "C" {

size_t gcdf_weight_count(const gcdf_net_desc* desc) {
  if (shape_check(desc) != GCDF_OK) return 0;
  return weight_count(desc->n_dof, desc->hidden, desc->n_hidden_layers);
}

int gcdf_create_net(const gcdf_net_desc* desc, const float* weights_host, size_t n_weights, gcdf_net** out) {
  int rc = shape_check(desc);
  if (rc) return rc;
  if (!weights_host || !out) return fail(GCDF_EINVAL, "weights_host or out is NULL");
  const size_t need = weight_count(desc->n_dof, desc->hidden, desc->n_hidden_layers);
  if (n_weights != need) return fail(GCDF_EINVAL, "n_weights %zu, shape needs %zu", n_weights, need);
  if (desc->precision == GCDF_FP32) {
    const int H = desc->hidden;
    if (H != 64 && H != 128 && H != 256 && H != 512)
      return fail(GCDF_EUNSUPPORTED, "FP32 path: hidden must be 64, 128, 256 or 512 (got %d)", H);
    if ((int)fp32_smem_bytes(H, desc->n_hidden_layers) > kSmemLimit)
      return fail(GCDF_EUNSUPPORTED, "FP32 path: %d layers of width %d exceed shared memory", desc->n_hidden_layers, H);
  } else if (!tc_supported(desc->hidden, desc->n_hidden_layers, desc->n_dof)) {
    return fail(GCDF_EUNSUPPORTED, "tensor-core path: shape (hidden %d, layers %d, n_dof %d) not built",
                desc->hidden, desc->n_hidden_layers, desc->n_dof);
  }
  gcdf_net* n = new (std::nothrow) gcdf_net();
  if (!n) return fail(GCDF_ENOMEM, "host allocation failed");
  memset(n, 0, sizeof(*n));
  n->n_dof = desc->n_dof;
  n->H = desc->hidden;
  n->L = desc->n_hidden_layers;
  n->precision = desc->precision;
  n->d_q = 2 + 2 * (desc->n_dof - 2);
  n->d_in = 3 + n->d_q;
  cudaError_t e = cudaGetDevice(&n->device);
  if (e != cudaSuccess) { free_net(n); return cuda_fail(e, "cudaGetDevice"); }
  e = cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, n->device);
  if (e != cudaSuccess) { free_net(n); return cuda_fail(e, "cudaDeviceGetAttribute"); }
  n->off_W1 = 0;
  n->off_b1 = (size_t)n->H * n->d_in;
  n->off_wout = need - 1 - n->H;
  n->bout = weights_host[need - 1];
  n->active_set = 1;
  if ((rc = dev_alloc_copy(&n->w_dev, weights_host, need))) { free_net(n); return rc; }
  {
    const int zero = 0;
    if ((rc = dev_alloc_copy(&n->err_word, &zero, 1))) { free_net(n); return rc; }
  }
  rc = (n->precision == GCDF_FP32) ? build_fp32_images(n, weights_host) : build_tc_images(n, weights_host);
  if (rc) { free_net(n); return rc; }
  *out = n;
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_destroy_net(gcdf_net* net) {
  if (!net) return GCDF_OK;
  cudaDeviceSynchronize();
  free_net(net);
  return GCDF_OK;
}

int gcdf_query(gcdf_net* net, const float* q, int N, const float* p, int M, const int* part_offsets,
               const int* part_idx, int n_pairs, const float* shift, float* f, float* grad,
               gcdf_stream_t stream) {
  WorkDesc w;
  int rc = check_call(net, q, N, p, M, part_offsets, part_idx, n_pairs, shift, w);
  if (rc) return rc;
  if (N == 0 || w.n_pairs == 0) return GCDF_OK;
  if (!f || !aligned16(f)) return fail(GCDF_EINVAL, "f is NULL or not 16-byte aligned");
  if (grad && !aligned16(grad)) return fail(GCDF_EINVAL, "grad not 16-byte aligned");
  w.mode = kQuery;
  w.f_out = f;
  w.g_out = grad;
  cudaStream_t s = (cudaStream_t)stream;
  Temps tmp(s);
  rc = run(net, w, shift, tmp, s);
  if (rc) return rc;
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_project(gcdf_net* net, const float* q, int N, const float* p, int M, const int* part_offsets,
                 const int* part_idx, int n_pairs, const float* shift, const float* m_diag, float* q_out,
                 gcdf_stream_t stream) {
  WorkDesc w;
  int rc = check_call(net, q, N, p, M, part_offsets, part_idx, n_pairs, shift, w);
  if (rc) return rc;
  if (N == 0 || w.n_pairs == 0) return GCDF_OK;
  if (!q_out || !aligned16(q_out)) return fail(GCDF_EINVAL, "q_out is NULL or not 16-byte aligned");
  if (m_diag && !aligned16(m_diag)) return fail(GCDF_EINVAL, "m_diag not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Temps tmp(s);
  cudaError_t e;
  float* f = nullptr;
  if ((e = tmp.get((void**)&f, (size_t)w.n_pairs * sizeof(float)))) return cuda_fail(e, "cudaMallocAsync");
  w.mode = kQuery;
  w.f_out = f;
  w.g_out = q_out;  // df/dq lands in q_out and is turned into q_z in place
  rc = run(net, w, shift, tmp, s);
  if (rc) return rc;
  if ((e = launch_project(q, N, net->n_dof, part_offsets, M, w.n_pairs, f, m_diag, q_out, s)))
    return cuda_fail(e, "projection launch");
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_collision_cost(gcdf_net* net, const float* q, int N, const float* p, int M, const int* part_offsets,
                        const int* part_idx, int n_pairs, const float* shift, int reduction, float param,
                        float* cost, float* grad, int* argmin, gcdf_stream_t stream) {
  WorkDesc w;
  int rc = check_call(net, q, N, p, M, part_offsets, part_idx, n_pairs, shift, w);
  if (rc) return rc;
  if (reduction != GCDF_RED_MIN && reduction != GCDF_RED_SOFTMIN && reduction != GCDF_RED_HINGE)
    return fail(GCDF_EINVAL, "unknown reduction %d", reduction);
  if (reduction == GCDF_RED_SOFTMIN && !(param > 0.f)) return fail(GCDF_EINVAL, "soft-min temperature must be > 0");
  if (reduction == GCDF_RED_HINGE && !(param == param)) return fail(GCDF_EINVAL, "hinge margin is NaN");
  if (N == 0) return GCDF_OK;
  if (!cost || !aligned16(cost) || !grad || !aligned16(grad))
    return fail(GCDF_EINVAL, "cost / grad NULL or not 16-byte aligned");
  if (argmin && !aligned16(argmin)) return fail(GCDF_EINVAL, "argmin not 16-byte aligned");
  w.mode = reduction;
  w.param = param;
  rc = reduce_call(net, w, shift, cost, grad, argmin, (cudaStream_t)stream);
  if (rc) return rc;
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_device_status(gcdf_net* net, int* status) {
  if (!net || !status) return fail(GCDF_EINVAL, "net or status is NULL");
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  if ((e = cudaMemcpy(&v, net->err_word, sizeof(int), cudaMemcpyDeviceToHost))) return cuda_fail(e, "cudaMemcpy");
  const int zero = 0;
  if ((e = cudaMemcpy(net->err_word, &zero, sizeof(int), cudaMemcpyHostToDevice))) return cuda_fail(e, "cudaMemcpy");
  *status = v;
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_set_active_set(gcdf_net* net, int enable) {
  if (!net) return fail(GCDF_EINVAL, "net is NULL");
  net->active_set = enable ? 1 : 0;
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_set_profile_events(gcdf_net* net, void* start_event, void* stop_event) {
  if (!net) return fail(GCDF_EINVAL, "net is NULL");
  if ((start_event == nullptr) != (stop_event == nullptr))
    return fail(GCDF_EINVAL, "give both profile events or neither");
  net->prof_start = (cudaEvent_t)start_event;
  net->prof_stop = (cudaEvent_t)stop_event;
  g_err[0] = 0;
  return GCDF_OK;
}

int gcdf_selftest_wait_expiry(gcdf_net* net, long long limit_cycles, int* seen) {
  if (!net || !seen) return fail(GCDF_EINVAL, "net or seen is NULL");
  if (limit_cycles < 1000 || limit_cycles > 4000000000LL)
    return fail(GCDF_EINVAL, "limit_cycles %lld outside [1e3, 4e9]", limit_cycles);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != net->device) return fail(GCDF_EINVAL, "net belongs to device %d, current device is %d", net->device, dev);
  int* d_seen = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_seen, 4 * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if ((e = cudaMemset(d_seen, 0xff, 4 * sizeof(int))) == cudaSuccess &&
      (e = launch_wait_expiry_probe(net->err_word, limit_cycles, d_seen, nullptr)) == cudaSuccess &&
      (e = cudaDeviceSynchronize()) == cudaSuccess)
    e = cudaMemcpy(seen, d_seen, 3 * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_seen);
  if (e != cudaSuccess) return cuda_fail(e, "wait-expiry self-test");
  g_err[0] = 0;
  return GCDF_OK;
}

long long gcdf_diag_fp32_fma(int blocks, int threads, int iters, float* sink, gcdf_stream_t stream) {
  if (blocks <= 0 || threads <= 0 || threads > 1024 || threads % 32 || iters <= 0 || !sink) {
    fail(GCDF_EINVAL, "bad FMA-loop arguments (blocks %d, threads %d, iters %d)", blocks, threads, iters);
    return -GCDF_EINVAL;
  }
  cudaError_t e = launch_fma_rate(blocks, threads, iters, sink, (cudaStream_t)stream);
  if (e != cudaSuccess) return -cuda_fail(e, "FMA loop launch");
  g_err[0] = 0;
  return (long long)blocks * threads * fma_rate_flops_per_thread(iters);
}

int gcdf_release_cached_memory(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return GCDF_OK;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    pool = g_pools[dev];
  }
  if (pool && (e = cudaMemPoolTrimTo(pool, 0)) != cudaSuccess) return cuda_fail(e, "cudaMemPoolTrimTo");
  g_err[0] = 0;
  return GCDF_OK;
}

const char* gcdf_last_error(void) { return g_err; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Collision cost without any allocation (gcdf_collision_cost_noalloc).
//
// Some callers must not allocate device memory once they are running: a
// trajectory optimizer inside a real-time control loop, where cudaMalloc /
// cudaMallocAsync can block, synchronise or fail at an unpredictable moment;
// a host application whose GPU memory is budgeted up front by another
// framework; or code that is certified to allocate only at start-up.  For
// them this entry point takes every temporary of a collision-cost call from
// one array that is part of the loaded library image on each device.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoAllocScratchBytes = 96u << 20;  // 96 MiB per device, held until the process exits
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array in the current device's context.  The
// host-side name of the array is not a device address.  Looked up on every
// call: the lookup is cheap once the module is loaded on the device, and a
// cached address would go stale if the context were destroyed and recreated
// (cudaDeviceReset), after which the array lives elsewhere.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
  *out = p;
  return GCDF_OK;
}

}  // namespace

extern "C" {

int gcdf_collision_cost_noalloc(gcdf_net* net, const float* q, int N, const float* p, int M,
                                const int* part_offsets, const int* part_idx, int n_pairs, const float* shift,
                                int reduction, float param, float* cost, float* grad, int* argmin,
                                gcdf_stream_t stream) {
  WorkDesc w;
  int rc = check_call(net, q, N, p, M, part_offsets, part_idx, n_pairs, shift, w);
  if (rc) return rc;
  if (reduction != GCDF_RED_MIN && reduction != GCDF_RED_SOFTMIN && reduction != GCDF_RED_HINGE)
    return fail(GCDF_EINVAL, "unknown reduction %d", reduction);
  if (reduction == GCDF_RED_SOFTMIN && !(param > 0.f)) return fail(GCDF_EINVAL, "soft-min temperature must be > 0");
  if (reduction == GCDF_RED_HINGE && !(param == param)) return fail(GCDF_EINVAL, "hinge margin is NaN");
  if (N == 0) return GCDF_OK;
  if (!cost || !aligned16(cost) || !grad || !aligned16(grad))
    return fail(GCDF_EINVAL, "cost / grad NULL or not 16-byte aligned");
  if (argmin && !aligned16(argmin)) return fail(GCDF_EINVAL, "argmin not 16-byte aligned");
  w.mode = reduction;
  w.param = param;

  // scratch layout: first-layer waypoint term, sin/cos, tile prefix (point
  // lists only), per-tile partial records; each part 256-byte aligned
  const size_t b_A = round256((size_t)N * net->H * sizeof(float));
  const size_t b_trig = round256((size_t)N * 2 * w.n_ang * sizeof(float));
  const size_t b_ts = part_offsets ? round256((size_t)(N + 1) * sizeof(int)) : 0;
  const size_t b_part = round256((size_t)(w.n_tiles > 0 ? w.n_tiles : 1) * sizeof(Partial));
  // the tensor-core kernel's stash of 2 s'(z_l) (per CTA, at most one CTA per SM)
  const size_t b_stash = net->precision == GCDF_FP32 ? 0 : round256(tc_stash_bytes(net->L, net->num_sms));
  const size_t need = b_A + b_trig + b_ts + b_part + b_stash;
  if (need > kNoAllocScratchBytes)
    return fail(GCDF_EINVAL,
                "request needs %zu bytes of scratch; the allocation-free entry point has %zu "
                "(use gcdf_collision_cost, or split the waypoints into smaller calls)",
                need, kNoAllocScratchBytes);
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  unsigned char* sp = static_cast<unsigned char*>(scratch);
  float* A = reinterpret_cast<float*>(sp);
  float* trig = reinterpret_cast<float*>(sp + b_A);
  int* ts = part_offsets ? reinterpret_cast<int*>(sp + b_A + b_trig) : nullptr;
  Partial* parts = reinterpret_cast<Partial*>(sp + b_A + b_trig + b_ts);
  w.A = A;
  w.trig = trig;
  w.partials = parts;
  w.stash = b_stash ? sp + b_A + b_trig + b_ts + b_part : nullptr;

  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (part_offsets) {
    if ((e = launch_tile_map(part_offsets, N, w.tile, ts, s))) return cuda_fail(e, "tile map launch");
    w.tile_start = ts;
  }
  if (w.n_pairs > 0) {
    if ((e = launch_prep(w, net->w_dev + net->off_W1, net->w_dev + net->off_b1, net->H, net->d_in, shift, A, trig,
                         s)))
      return cuda_fail(e, "prep launch");
    if (net->prof_start && (e = cudaEventRecord(net->prof_start, s))) return cuda_fail(e, "cudaEventRecord");
    if (net->precision == GCDF_FP32) {
      Fp32Weights fw;
      fw.BF = net->BF;
      fw.BB = net->BB;
      fw.bias = net->bias_p;
      fw.W1 = net->w_dev + net->off_W1;
      fw.wout = net->wout_p;
      fw.bout = net->bout;
      fw.H = net->H;
      fw.L = net->L;
      fw.d_in = net->d_in;
      fw.d_q = net->d_q;
      if ((e = launch_fp32(w, fw, net->num_sms, s))) return cuda_fail(e, "fp32 kernel launch");
    } else {
      if ((e = launch_tc(w, net->tcw, net->num_sms, s))) return cuda_fail(e, "tensor-core kernel launch");
    }
    if (net->prof_stop && (e = cudaEventRecord(net->prof_stop, s))) return cuda_fail(e, "cudaEventRecord");
  } else if (!part_offsets) {
    w.tiles_per_wp = 0;
  }
  if ((e = launch_merge(w, N, cost, grad, argmin, s))) return cuda_fail(e, "merge launch");
  g_err[0] = 0;
  return GCDF_OK;
}

}  // extern "C"
