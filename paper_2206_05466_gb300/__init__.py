"""Zeitlin-Euler IsoMP hot path on GB300 (sm_103a)."""
