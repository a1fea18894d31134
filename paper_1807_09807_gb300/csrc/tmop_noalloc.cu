// tmop_energy_noalloc: the FP64 objective and minimum det A of a structured
// order-k grid, computed without any device allocation.
//
// Who needs it: callers that are not allowed to allocate GPU memory at the
// point where they evaluate mesh quality -- for example a host application
// whose own device allocator owns the whole GPU (an arena or pool that a
// stray cudaMalloc would fragment or overrun), a plugin called from inside
// another code's time step where cudaMalloc's implicit synchronisation is not
// acceptable, or a caller that cannot keep a tmop_setup context alive. They
// pass the positions and two device scalars for the results; everything
// else the call needs lives in this file.
//
// The element kernel is the same one tmop_energy launches (one warp per
// element); only its scratch differs: the per-block partial sums of F and of
// min det A go into the file-scope array below instead of a context's
// workspace, and the launch uses one block per group of `warps` elements
// (4 to 8), so the number of partials is ceil(nelem / warps).
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>
#include <stdint.h>
#include <string.h>

#include "../../include/tmop.h"
#include "tmop_kparams.h"
#include "tmop_vec.h"

namespace tmop {

// Partial sums: [0, kNoAllocMaxBlocks) for F, [kNoAllocMaxBlocks, 2x) for
// min det A. 2 x 32768 doubles = 512 KiB, held by every GPU that loads the
// library until the process exits.
constexpr int kNoAllocMaxBlocks = 32768;
static __device__ __align__(256) double g_noalloc_partials[2 * kNoAllocMaxBlocks];

constexpr int kMaxDevices = 64;
static double* g_partials_addr[kMaxDevices];  // device address of the array, per device
static std::mutex g_setup_mutex;

// Once per device, with that device current: the host-side name of a
// __device__ array is only a stand-in, so the kernel must be given the
// address the runtime reports for the current device.
static int partials_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TMOP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) return TMOP_ERR_CUDA;
    g_partials_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_partials_addr[dev];
  return TMOP_OK;
}

}  // namespace tmop

using namespace tmop;

extern "C" int tmop_energy_noalloc(int dim, int order, const int structured[3], const tmop_quad* quad,
                                   int metric_id, const tmop_targets* targets, const double* x, double* F,
                                   double* min_detA, void* stream) {
  if (!structured || !quad || !targets || !x || !F || !min_detA) return TMOP_ERR_ARG;
  if (dim != 2 && dim != 3) return TMOP_ERR_ARG;
  if (order < 1 || order > 4) return TMOP_ERR_ARG;
  if (quad->kind != TMOP_GL && quad->kind != TMOP_GLL) return TMOP_ERR_ARG;
  if (quad->npts1d < 2 || quad->npts1d > kMaxQ) return TMOP_ERR_ARG;
  const bool ok_metric = metric_supported(dim, metric_id);
  if (!ok_metric) return TMOP_ERR_ARG;
  const int nx = structured[0], ny = structured[1], nz = dim == 3 ? structured[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1) return TMOP_ERR_ARG;
  const long long nelem = (long long)nx * ny * nz;
  const long long nnode = (long long)(order * nx + 1) * (order * ny + 1) * (dim == 3 ? order * nz + 1 : 1);
  if (nelem > 0x7fffffffLL || nnode > 0x7fffffffLL) return TMOP_ERR_ARG;
  const int n = order + 1, nq = quad->npts1d;
  const ElemEntry* ent = find_elem(dim, n, nq, 0, OP_ENERGY);
  if (!ent) return TMOP_ERR_ARG;
  const long long blocks = (nelem + ent->warps - 1) / ent->warps;
  if (blocks > kNoAllocMaxBlocks) return TMOP_ERR_CAPACITY;

  KParams p;
  memset(&p, 0, sizeof(p));
  p.dim = dim;
  p.nelem = (int)nelem;
  p.nnode = (int)nnode;
  p.metric = metric_id;
  p.sx = nx; p.sy = ny; p.sz = dim == 3 ? nz : 0;
  double qx[kMaxQ], qw[kMaxQ], z[kMaxN], zw[kMaxN];
  if (quad->kind == TMOP_GL) rule_gl(nq, qx, qw);
  else rule_gll(nq, qx, qw);
  rule_gll(n, z, zw);
  for (int a = 0; a < nq; ++a) {
    double phi[kMaxN], dphi[kMaxN];
    lagrange_bary(n, z, qx[a], phi, dphi);
    for (int i = 0; i < n; ++i) {
      p.B[a * n + i] = phi[i];
      p.G[a * n + i] = dphi[i];
    }
    p.w1[a] = qw[a];
  }
  double Wc[9] = {0};
  switch (targets->kind) {
    case TMOP_W_IDENTITY:
      for (int i = 0; i < dim; ++i) Wc[i * dim + i] = 1.0;
      p.wkind = WK_IDENTITY;
      break;
    case TMOP_W_SCALED:
      if (!(targets->scale > 0.0) || !isfinite(targets->scale)) return TMOP_ERR_ARG;
      for (int i = 0; i < dim; ++i) Wc[i * dim + i] = targets->scale;
      p.wkind = WK_CONST;
      break;
    case TMOP_W_CONST:
      if (!targets->W) return TMOP_ERR_ARG;
      memcpy(Wc, targets->W, sizeof(double) * dim * dim);
      p.wkind = WK_CONST;
      break;
    default:  // per-point targets would need a device copy of W^-1
      return TMOP_ERR_ARG;
  }
  if (!inv_h(dim, Wc, p.Winv, &p.detW)) return TMOP_ERR_ARG;

  double* partials = nullptr;
  int rc = partials_for_current_device(&partials);
  if (rc != TMOP_OK) return rc;
  // Every block writes its own partial, and the final pass reads only the
  // first `blocks` of them, so nothing left by an earlier call needs clearing.
  p.part_F = partials;
  p.part_min = partials + kNoAllocMaxBlocks;
  p.x = x;
  int grid = 0;
  if (ent->prepare((int)nelem, &grid) != 0) return TMOP_ERR_CUDA;  // shared-memory opt-in only
  cudaStream_t s = (cudaStream_t)stream;
  if (ent->launch(p, (int)blocks, s) != 0) return TMOP_ERR_CUDA;
  if (energy_final(p.part_F, p.part_min, (int)blocks, nullptr, 0, F, min_detA, s) != 0) return TMOP_ERR_CUDA;
  return TMOP_OK;
}
