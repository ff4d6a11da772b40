"""GB300-native loss-and-gradient engine for Adorym's multislice ptychography forward model.

The compute path lives in ``libadorym.so`` (hand-written sm_103a CUDA behind
a C ABI, ``include/adorym.h``); ``adorym`` is its ctypes binding and
``autograd`` wraps it in a ``torch.autograd.Function``.  ``synth`` draws the
seeded synthetic inputs.  Submodules are imported lazily so that ``synth``
can be used without the library.
"""
