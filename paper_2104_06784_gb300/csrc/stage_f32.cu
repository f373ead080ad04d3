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
int launch_stage_batch<float>(const StageArgs<float> *args_device, int nsim, const BatchStrip *strips_device, int nstrips,
                            BatchTile *list, unsigned int *list_n, void *stream)
{
    return launch_stage_batch_impl<float>(args_device, nsim, strips_device, nstrips, list, list_n, stream);
}

}  // namespace moses
