"""Seeded synthetic workloads (input generators only; no clustering arithmetic)."""
from .generators import *  # noqa: F401,F403
