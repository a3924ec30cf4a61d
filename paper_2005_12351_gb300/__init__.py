"""GB300-native (sm_103a) Cartesian-Taylor FMM for point sources of any order.

Implements the evaluation path of Pepper & Fangohr, "fmmgen" (arXiv:2005.12351):
octree, P2M/M2M, M2L over dual-tree interaction lists, L2L/L2P and the P2P
near field, as hand-written CUDA behind the C ABI in include/fmm_gb300.h.

    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=128)
    tree.set_sources(pos, moments, source_order=1)     # CUDA float64 tensors
    phi, E = tree.evaluate(p=6, theta=0.5)

``synth`` draws the seeded synthetic workloads.  ``fmm`` needs the built
extension (``__graft_entry__.build()``); there is no CPU fallback.
"""
__all__ = ["fmm", "synth", "build"]
