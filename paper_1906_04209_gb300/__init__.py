"""GB300-native fast solver for the narrow capture / narrow escape problems on
the sphere (Kaye & Greengard). The compute path lives in the CUDA library
``csrc/`` builds; ``ncs`` is its thin ctypes binding and ``layouts`` holds the
seeded synthetic patch layouts. Importing the package loads nothing native."""
