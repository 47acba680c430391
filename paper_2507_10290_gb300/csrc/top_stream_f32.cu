// FP32 instantiation of the streaming CADMM form.
#include "top_stream.cuh"

namespace top {
int launch_stream_f32(const StreamArgs &a, int fam, void *stream) { return run_stream_t<float>(a, fam, stream); }
}  // namespace top
