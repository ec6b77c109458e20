"""GB300 (sm_103a) two-link staggered quark smearing (arXiv:2301.05518).

The compute path is the CUDA library ``libtls.so`` behind the C ABI in
``include/tls.h``; ``paper_2301_05518_gb300.tls`` is its Python binding and
``paper_2301_05518_gb300.synth`` draws seeded synthetic inputs.  Importing the
package itself loads nothing; ``from paper_2301_05518_gb300 import tls`` loads
the library and fails loudly if it has not been built.
"""

__all__ = ["tls", "synth", "build"]
