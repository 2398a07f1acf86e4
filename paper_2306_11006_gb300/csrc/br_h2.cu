// br_h2.cu -- blind-rotation kernel shapes with H = 2 (2H warps per gate).
#include "br_kernel.cuh"

namespace arx {

cudaError_t launch_br_h2(const BrArgs &args, int GT, int grid, cudaStream_t st) {
  switch (GT) {
    case 1: return br::launch_shape<2, 1>(args, grid, st);
    case 3: return br::launch_shape<2, 3>(args, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t br_smem_h2(int GT) {
  switch (GT) {
    case 1: return br::br_smem_bytes<2, 1>();
    case 3: return br::br_smem_bytes<2, 3>();
    default: return 0;
  }
}

int br_occupancy_h2(int GT) {
  switch (GT) {
    case 1: return br::occupancy_shape<2, 1>();
    case 3: return br::occupancy_shape<2, 3>();
    default: return 0;
  }
}

}  // namespace arx
