// engine_f64.cu -- the pipeline instantiated for the plain FP64 position form.
#include "engine_impl.cuh"

namespace dem {
EngineBase *make_engine_f64() { return new Engine<FormF64>(); }
}  // namespace dem
