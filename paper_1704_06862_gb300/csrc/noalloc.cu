// Allocation-free variant of the ILU(0) apply.
//
// ilu_apply() stages its vectors in work buffers the context allocates on
// first use (cudaMalloc).  Some callers cannot let a library allocate device
// memory during a step: for example code that runs under a host framework
// owning every device allocation through its own pool, or a latency-critical
// loop in which a cudaMalloc would synchronise the device.  This entry point
// does the same work with its scratch taken from a fixed, file-scope device
// array instead, and allocates nothing.
#include <mutex>

#include "common.h"

namespace {

// Scratch of the allocation-free apply: the two internal-order complex128
// vectors and their complex64 copies, [nrhs][n_rwg][2] each.  Every GPU that
// loads the library holds this array until the process exits.
constexpr size_t kNoAllocBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array, looked up once per device (host code cannot
// use the symbol itself: on the host it is only a stand-in).
constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

void *scratch_for(int device) {
  SIE_REQUIRE(device >= 0 && device < kMaxDevices, SIE_EINVAL, "ilu_apply_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    SIE_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[device] = p;
  }
  return g_scratch_ptr[device];
}

}  // namespace

extern "C" sie_status ilu_apply_noalloc(sie_ctx *c, const void *r, void *z, int64_t nrhs, sie_prec prec) {
  if (!c) return SIE_EINVAL;
  try {
    SIE_CUDA(cudaSetDevice(c->device));
    SIE_REQUIRE(c->have_fill && c->ilu.ready, SIE_ESTATE, "ilu_apply_noalloc: no ILU factors (fill with build_ilu)");
    SIE_REQUIRE(r && z && r != z && nrhs >= 1, SIE_EINVAL, "ilu_apply_noalloc: bad buffers or nrhs");
    SIE_REQUIRE(prec == SIE_PREC_FP64 || prec == SIE_PREC_MIXED, SIE_EINVAL, "ilu_apply_noalloc: bad precision");
    const size_t n = (size_t)nrhs * c->ne * 2;  // complex entries per vector
    const size_t need = n * (2 * sizeof(zd) + 2 * sizeof(zf));
    SIE_REQUIRE(need <= kNoAllocBytes, SIE_EINVAL,
                "ilu_apply_noalloc: nrhs * n_rwg exceeds the 16 MiB scratch (limit nrhs * n_rwg <= 174762)");
    unsigned char *base = (unsigned char *)scratch_for(c->device);
    zd *xi = (zd *)base;
    zd *yi = xi + n;
    zf *xf = (zf *)(yi + n);
    zf *yf = xf + n;
    // every element of the outputs below is written before it is read: no clearing needed
    op_permute_in(c, (const zd *)r, xi, (int)nrhs);
    if (prec == SIE_PREC_FP64) {
      op_ilu<double>(c, xi, yi, (int)nrhs);
    } else {
      op_d2f(c, xi, xf, (int64_t)n);
      op_ilu<float>(c, xf, yf, (int)nrhs);
      op_f2d(c, yf, yi, (int64_t)n);
    }
    op_permute_out(c, yi, (zd *)z, (int)nrhs);
    return SIE_OK;
  } catch (const SieError &e) {
    c->last_error = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    c->last_error = e.what();
    return SIE_EINVAL;
  }
}
