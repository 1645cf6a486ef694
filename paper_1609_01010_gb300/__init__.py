"""GB300-native exact polynomial multiplication over Z/pZ through the TFT.

The compute path is the CUDA shared library ``libpolymul.so`` (built from
``csrc/`` for sm_103a) behind a C ABI declared in ``include/polymul.h``;
``binding`` marshals arguments to it and nothing else.  Importing this package
does not load the library; ``binding.lib()`` does, and fails loudly when it is
missing.
"""
