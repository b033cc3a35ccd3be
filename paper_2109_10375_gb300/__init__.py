"""GB300-native reionization-redshift assignment z_re(x) of AMBER (arXiv 2109.10375).

The compute path lives in the CUDA library libamber.so (C ABI in include/amber.h);
``binding`` marshals torch tensors to it.  ``synth`` makes seeded input fields.
"""
