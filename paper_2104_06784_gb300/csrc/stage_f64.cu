// stage_f64.cu -- the stage kernels and their launchers for the double element type.
#include "stage_launch.cuh"

namespace moses {

template <>
int launch_stage<double>(const StageArgs<double> &a, int tile, void *stream)
{
    return launch_stage_impl<double>(a, tile, stream);
}

template <>
int launch_stage_rec<double>(const StageArgs<double> &a, void *stream)
{
    return launch_stage_rec_impl<double>(a, stream);
}

template <>
int launch_batch<double>(const BatchRun<double> &r, int ty, int *grid, void *stream)
{
    return launch_batch_impl<double>(r, ty, grid, stream);
}

}  // namespace moses
