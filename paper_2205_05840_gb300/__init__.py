"""GB300-native V-cycle multigrid for lowest-order hexahedral Nedelec H(curl)
problems with nonoverlapping domain-decomposition smoothers (arXiv 2205.05840).

The compute path is the C-ABI library ``libndmg.so`` (CUDA, sm_103a); the
Python side only marshals arguments.  ``import paper_2205_05840_gb300.ndmg``
loads the library and fails loudly if it has not been built.
"""
