// The library's capture guard (host only).  Capturing a CUDA graph on one thread is invalidated by
// device-wide calls of other threads (a device synchronisation, a free, a synchronous copy or memset, a
// first-time module load or symbol lookup).  Every library call that makes such calls holds this guard
// shared; a graph capture holds it exclusively.
#pragma once
#include <shared_mutex>

namespace bura {
std::shared_mutex& capture_guard();
}  // namespace bura
