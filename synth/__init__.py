"""Seeded synthetic fragment pairs shaped like RGB-D TSDF / surfel scene fragments.

This module only makes inputs: scene geometry, point sampling, rigid motions,
cropping, noise and outliers. It holds none of the registration arithmetic,
and both the CUDA path's tests/bench and the oracle's tests draw from it.
"""
from .fragments import (CONFIGS, FragmentPair, make_pair, make_batch, random_rotation, random_pose,  # noqa: F401
                        pose_error)
