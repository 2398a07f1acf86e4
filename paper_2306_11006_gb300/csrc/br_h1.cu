// br_h1.cu -- blind-rotation kernel shapes with H = 1 (2H warps per gate).
#include "br_kernel.cuh"

namespace arx {

cudaError_t launch_br_h1(const BrArgs &args, int GT, int grid, cudaStream_t st) {
  switch (GT) {
    case 1: return br::launch_shape<1, 1>(args, grid, st);
    case 2: return br::launch_shape<1, 2>(args, grid, st);
    case 4: return br::launch_shape<1, 4>(args, grid, st);
    case 6: return br::launch_shape<1, 6>(args, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t br_smem_h1(int GT) {
  switch (GT) {
    case 1: return br::br_smem_bytes<1, 1>();
    case 2: return br::br_smem_bytes<1, 2>();
    case 4: return br::br_smem_bytes<1, 4>();
    case 6: return br::br_smem_bytes<1, 6>();
    default: return 0;
  }
}

int br_occupancy_h1(int GT) {
  switch (GT) {
    case 1: return br::occupancy_shape<1, 1>();
    case 2: return br::occupancy_shape<1, 2>();
    case 4: return br::occupancy_shape<1, 4>();
    case 6: return br::occupancy_shape<1, 6>();
    default: return 0;
  }
}

}  // namespace arx
