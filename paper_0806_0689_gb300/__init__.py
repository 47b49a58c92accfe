"""GB300-native block-matching motion estimation (DCDS and full search)."""
