"""GB300-native generalized Sinkhorn scaling for entropic unbalanced optimal transport.

Chizat, Peyre, Schmitzer, Vialard, "Scaling algorithms for unbalanced optimal
transport problems" (arXiv:1607.05816): the scaling iterations (S) of Sec. 3.3,
run in the log domain of Sec. 4.3 (Algorithm 2 with absorption), with the
proxdiv operators of Table 1 and the barycenter operators of Table 2.

The compute path is the C-ABI library ``libuot.so`` (see ``include/uot.h``);
``paper_1607_05816_gb300.uot`` is its thin ctypes binding.  Importing this
package does not load the library; ``synth`` only generates seeded inputs.
"""

__all__ = ["synth", "uot"]
