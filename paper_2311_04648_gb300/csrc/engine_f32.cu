// engine_f32.cu -- the pipeline instantiated for the voxel-index + FP32-offset form.
#include "engine_impl.cuh"

namespace dem {
EngineBase *make_engine_f32() { return new Engine<FormF32>(); }
}  // namespace dem
