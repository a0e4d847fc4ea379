// Dispatch of a PCG launch to the instantiation for its nx.
#include "kernels.h"

namespace sspcg {

cudaError_t launch_pcg_nx1(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx2(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx3(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx4(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx5(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx6(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx7(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx8(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx9(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx10(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx11(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx12(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx13(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx14(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx15(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx16(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx17(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx18(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx19(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx20(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx21(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx22(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx23(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx24(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx25(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx26(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx27(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_pcg_nx28(int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem, cudaStream_t st);

cudaError_t launch_pcg(int nx, int op, int red, bool f64, const PcgArgs &a, int grid, int block, size_t smem,
                       cudaStream_t st) {
  switch (nx) {
    case 1: return launch_pcg_nx1(op, red, f64, a, grid, block, smem, st);
    case 2: return launch_pcg_nx2(op, red, f64, a, grid, block, smem, st);
    case 3: return launch_pcg_nx3(op, red, f64, a, grid, block, smem, st);
    case 4: return launch_pcg_nx4(op, red, f64, a, grid, block, smem, st);
    case 5: return launch_pcg_nx5(op, red, f64, a, grid, block, smem, st);
    case 6: return launch_pcg_nx6(op, red, f64, a, grid, block, smem, st);
    case 7: return launch_pcg_nx7(op, red, f64, a, grid, block, smem, st);
    case 8: return launch_pcg_nx8(op, red, f64, a, grid, block, smem, st);
    case 9: return launch_pcg_nx9(op, red, f64, a, grid, block, smem, st);
    case 10: return launch_pcg_nx10(op, red, f64, a, grid, block, smem, st);
    case 11: return launch_pcg_nx11(op, red, f64, a, grid, block, smem, st);
    case 12: return launch_pcg_nx12(op, red, f64, a, grid, block, smem, st);
    case 13: return launch_pcg_nx13(op, red, f64, a, grid, block, smem, st);
    case 14: return launch_pcg_nx14(op, red, f64, a, grid, block, smem, st);
    case 15: return launch_pcg_nx15(op, red, f64, a, grid, block, smem, st);
    case 16: return launch_pcg_nx16(op, red, f64, a, grid, block, smem, st);
    case 17: return launch_pcg_nx17(op, red, f64, a, grid, block, smem, st);
    case 18: return launch_pcg_nx18(op, red, f64, a, grid, block, smem, st);
    case 19: return launch_pcg_nx19(op, red, f64, a, grid, block, smem, st);
    case 20: return launch_pcg_nx20(op, red, f64, a, grid, block, smem, st);
    case 21: return launch_pcg_nx21(op, red, f64, a, grid, block, smem, st);
    case 22: return launch_pcg_nx22(op, red, f64, a, grid, block, smem, st);
    case 23: return launch_pcg_nx23(op, red, f64, a, grid, block, smem, st);
    case 24: return launch_pcg_nx24(op, red, f64, a, grid, block, smem, st);
    case 25: return launch_pcg_nx25(op, red, f64, a, grid, block, smem, st);
    case 26: return launch_pcg_nx26(op, red, f64, a, grid, block, smem, st);
    case 27: return launch_pcg_nx27(op, red, f64, a, grid, block, smem, st);
    case 28: return launch_pcg_nx28(op, red, f64, a, grid, block, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t occupancy_pcg_nx1(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx2(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx3(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx4(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx5(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx6(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx7(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx8(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx9(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx10(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx11(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx12(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx13(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx14(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx15(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx16(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx17(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx18(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx19(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx20(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx21(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx22(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx23(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx24(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx25(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx26(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx27(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);
cudaError_t occupancy_pcg_nx28(int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas);

cudaError_t occupancy_pcg(int nx, int op, int red, bool f64, bool gv, bool cg, bool warp, int block, size_t smem, int *ctas) {
  switch (nx) {
    case 1: return occupancy_pcg_nx1(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 2: return occupancy_pcg_nx2(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 3: return occupancy_pcg_nx3(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 4: return occupancy_pcg_nx4(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 5: return occupancy_pcg_nx5(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 6: return occupancy_pcg_nx6(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 7: return occupancy_pcg_nx7(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 8: return occupancy_pcg_nx8(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 9: return occupancy_pcg_nx9(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 10: return occupancy_pcg_nx10(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 11: return occupancy_pcg_nx11(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 12: return occupancy_pcg_nx12(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 13: return occupancy_pcg_nx13(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 14: return occupancy_pcg_nx14(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 15: return occupancy_pcg_nx15(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 16: return occupancy_pcg_nx16(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 17: return occupancy_pcg_nx17(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 18: return occupancy_pcg_nx18(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 19: return occupancy_pcg_nx19(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 20: return occupancy_pcg_nx20(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 21: return occupancy_pcg_nx21(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 22: return occupancy_pcg_nx22(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 23: return occupancy_pcg_nx23(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 24: return occupancy_pcg_nx24(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 25: return occupancy_pcg_nx25(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 26: return occupancy_pcg_nx26(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 27: return occupancy_pcg_nx27(op, red, f64, gv, cg, warp, block, smem, ctas);
    case 28: return occupancy_pcg_nx28(op, red, f64, gv, cg, warp, block, smem, ctas);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sspcg
