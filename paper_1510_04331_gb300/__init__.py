"""GB300 (sm_103a) library for the data-parallel hot path of the GRAPHIC
angular-differential-imaging reduction (arXiv:1510.04331): Fourier
recentring shift, angle-gated median PSF subtraction, Fourier three-shear
derotation and median collapse, behind the C ABI of ``include/graphic.h``.

``paper_1510_04331_gb300.graphic`` is the ctypes binding (loaded on first
use; it raises ``GraphicError`` when the CUDA library is missing).
``paper_1510_04331_gb300.synth`` generates seeded synthetic ADI cubes.
"""

__all__ = ["graphic", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
