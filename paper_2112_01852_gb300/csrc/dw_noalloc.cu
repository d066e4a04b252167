// Allocation-free variant of dw_apply_DdagD.
//
// dw_apply_DdagD keeps the intermediate D in in lattice-owned scratch that it
// grows with cudaMalloc on first use.  Some callers cannot have the library
// allocate device memory behind their back: for instance a serving process
// whose device memory is entirely handed out by its own pool allocator, or a
// host that must not perform allocation calls while its work is in flight.
// For them dw_apply_DdagD_noalloc keeps the intermediate in one fixed array
// compiled into the library instead, and calls no allocation routine.
#include <mutex>

#include "dw_api_internal.cuh"

namespace dw {
namespace {

// One array per GPU that loads the library, held until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of the array on the current device (host code only holds a
// stand-in for the symbol, so the address is looked up once per device).
int scratch_address(int dev, void **ptr) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "address of the no-alloc scratch array");
    g_scratch_addr[dev] = p;
  }
  *ptr = g_scratch_addr[dev];
  return DW_OK;
}

}  // namespace
}  // namespace dw

using namespace dw;

extern "C" int dw_apply_DdagD_noalloc(dw_lattice *lat, void *out, const void *in,
                                      const double *mf, int nrhs, void *stream) {
  clear_error();
  int rc = check_apply(lat, out, in, mf, nrhs, true);
  if (rc) return rc;
  const size_t need = field_bytes(lat, lat->prec, nrhs);
  if (need > kNoAllocScratchBytes)
    return fail(DW_ERR_ARG,
                "dw_apply_DdagD_noalloc: %d RHS of this lattice need %zu bytes of scratch, more "
                "than the fixed %zu-byte array",
                nrhs, need, kNoAllocScratchBytes);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != lat->device)
    return fail(DW_ERR_ARG, "current device %d is not the lattice's device %d", dev, lat->device);
  if (dev < 0 || dev >= kMaxDevices) return fail(DW_ERR_ARG, "device index %d out of range", dev);
  void *scratch = nullptr;
  if ((rc = scratch_address(dev, &scratch))) return rc;
  // The D pass overwrites every element of the intermediate, so nothing in the
  // array needs clearing first.
  cudaStream_t st = (cudaStream_t)stream;
  rc = run_dslash(lat, lat->prec, OP_D, scratch, in, mf, nrhs, st, nullptr);
  if (rc) return rc;
  return run_dslash(lat, lat->prec, OP_DDAG, out, scratch, mf, nrhs, st, nullptr);
}
