"""GB300-native batched ray-cast depth / LiDAR renderer (placeholder; the binding lands with the CUDA library)."""
