// fc_cnn.cu -- learned refinement tagger kernels (BF16 weights, FP32 accumulation).
#include "fc_internal.cuh"

extern "C" {
int fc_cnn_forward(int, int, const float *, const float *, float *, void *)
{
    fc::set_error("learned tagger not built");
    return FC_ERR_UNIMPLEMENTED;
}
int fc_cnn_loss_grad(int, int, const float *, const float *, const float *, float *, float *, void *)
{
    fc::set_error("learned tagger not built");
    return FC_ERR_UNIMPLEMENTED;
}
int fc_cnn_adam(float *, const float *, float *, float *, int, float, void *)
{
    fc::set_error("learned tagger not built");
    return FC_ERR_UNIMPLEMENTED;
}
}
