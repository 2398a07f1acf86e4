// br_h4.cu -- blind-rotation kernel shapes with H = 4 (2H warps per gate); gadget length L = 2 only.
#include "br_kernel.cuh"

namespace arx {

cudaError_t launch_br_h4(const BrArgs &args, int GT, int L, int grid, cudaStream_t st) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::launch_shape<4, 1, 2>(args, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

size_t br_smem_h4(int GT, int L) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::br_smem_bytes<4, 1, 2>();
      default: return 0;
    }
  }
  return 0;
}

int br_occupancy_h4(int GT, int L) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::occupancy_shape<4, 1, 2>();
      default: return 0;
    }
  }
  return 0;
}

}  // namespace arx
