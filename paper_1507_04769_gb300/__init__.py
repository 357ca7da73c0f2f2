"""GB300 (sm_103a) implementation of the sparse grid characteristics method
for optimal feedback control (Kang & Wilcox): sparse-grid construction,
per-node characteristic BVP solves, hierarchical surpluses and on-line
feedback evaluation, behind the C ABI of include/sg.h.

The CUDA library is loaded by `paper_1507_04769_gb300.sg`; importing the
package itself does not touch the GPU.
"""
__all__ = ["sg", "build"]
