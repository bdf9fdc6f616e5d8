"""Seeded synthetic inputs for MRF reconstruction: flip-angle trains, Bloch-response
dictionaries, ellipse phantoms, Cartesian line masks, noise and the simulated acquisition.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's tests.  It holds
none of the reconstruction's arithmetic (no gradient step, no matched filter, no tree search):
it only synthesises data with the shapes and structure of the paper's experiments (§6).
Every random draw uses ``numpy.random.Generator(PCG64(seed))`` with the fixed seed scheme in
:mod:`mrfgen.configs`.
"""
from .sequence import flip_train, param_grid
from .bloch import epg_fisp, bssfp, simulate_dictionary
from .phantom import ellipse_phantom, line_masks, acquire
from .configs import CONFIGS, make_problem, make_dictionary, slice_geometry

__all__ = [
    "flip_train", "param_grid", "epg_fisp", "bssfp", "simulate_dictionary",
    "ellipse_phantom", "line_masks", "acquire", "CONFIGS", "make_problem", "make_dictionary",
    "slice_geometry",
]
