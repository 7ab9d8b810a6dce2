"""Guided walk on stars (arXiv 2410.18944) on one GB300: CUDA library
``libwost`` (include/wost.h) and its thin Python binding.

    from paper_2410_18944_gb300 import api
    sc = api.Scene(scene_description)
    mean, var, stats = api.solve(sc, points, nwalks=32, guided=False)
"""
__all__ = ["api", "build"]
