"""GB300 (sm_103a) implementation of the spatio-temporal dynamic-mesh codec of
"Fast Spatio-temporal Compression of Dynamic 3D Meshes" (Arvanitis, Lalos,
Moustakas).

The codec runs in ``libmesh_codec.so`` (CUDA, C ABI in
``include/mesh_codec.h``); ``codec`` is its ctypes binding.
"""

from .codec import MeshCodec, MeshCodecError, load_library, default_params  # noqa: F401
