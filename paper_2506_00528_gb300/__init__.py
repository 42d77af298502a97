"""GB300-native EVP ternary embedding search (arXiv 2506.00528).

The compute path lives in the CUDA library ``libevp.so`` (see ``csrc/``);
``evp`` holds its thin ctypes binding.  ``synth`` draws seeded inputs.
"""
