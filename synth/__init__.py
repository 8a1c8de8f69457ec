"""Seeded synthetic transit timetables and queries (inputs only; no method arithmetic)."""
from .transit import (  # noqa: F401
    CONFIGS, QuerySet, Timetable, city, grid_timetable, large, ragged_grids,
    random_queries, single_route, small_grid, tiny_random,
)
