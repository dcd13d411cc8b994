"""Proposal-network reference (filled in with the learned proposal)."""
__all__ = []
