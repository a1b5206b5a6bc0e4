"""GB300 (sm_103a) star-M truncated tensor SVD: mode-3 TTM, batched one-sided Jacobi slice
SVDs, t-SVDM-I / t-SVDM-II, reconstruction and the truncation-loss gradient, behind the C
ABI of libtsvdm.so (include/tsvdm.h).  Submodules load lazily: ``synth`` needs only NumPy;
``native`` and ``tsvdm`` need the built library and PyTorch."""

__all__ = ["native", "synth", "tsvdm", "build"]
