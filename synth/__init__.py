"""Seeded synthetic frame pairs shaped like driving scenes.

This package only draws inputs: textures, flow fields and noise. It holds none of
the arithmetic of DeGraF or RLOF, and both the CUDA path and the CPU oracle take
their inputs from it.
"""
from .pairs import (  # noqa: F401
    Pair,
    Texture,
    make_pair,
    make_translation_pair,
    make_radial_pair,
    make_batch_specs,
    CONFIG_SIZES,
    render,
    render_affine,
)
