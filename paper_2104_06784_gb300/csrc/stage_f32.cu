// stage_f32.cu -- the stage kernels and their launchers for the float element type.
#include "stage_launch.cuh"

namespace moses {

template <>
int launch_stage<float>(const StageArgs<float> &a, int tile, void *stream)
{
    return launch_stage_impl<float>(a, tile, stream);
}

template <>
int launch_stage_rec<float>(const StageArgs<float> &a, void *stream)
{
    return launch_stage_rec_impl<float>(a, stream);
}

template <>
int launch_batch<float>(const BatchRun<float> &r, int ty, int *grid, void *stream)
{
    return launch_batch_impl<float>(r, ty, grid, stream);
}

}  // namespace moses
