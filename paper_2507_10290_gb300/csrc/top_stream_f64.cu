// FP64 instantiation of the streaming CADMM form.
#include "top_stream.cuh"

namespace top {
int launch_stream_f64(const StreamArgs &a, int fam, void *stream) { return run_stream_t<double>(a, fam, stream); }
}  // namespace top
